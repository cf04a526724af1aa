// LDU face addressing -> block CSR (Sec. 2.3, Alg. 1: permute the matrix
// coefficients from LDU into block-CSR order).
//
// Structure (once per topology): row i of the block-CSR matrix holds the
// diagonal block and one block per face touching cell i, columns ascending.
// Every BSR position p records its LDU source src[p]:
//   -1 - i  diag[i]
//   2 f     upper[f]  (row owner[f], column neighbour[f])
//   2 f + 1 lower[f]  (row neighbour[f], column owner[f])
// Values (every nonlinear iteration): val[p] = source block, a pure gather
// with coalesced n*n-double writes.
#include <algorithm>

#include "internal.h"

namespace bcs {

namespace {

__global__ void k_check_count(int C, int F, const int32_t* __restrict__ owner,
                              const int32_t* __restrict__ nb, int32_t* __restrict__ cnt,
                              int32_t* __restrict__ err) {
  dep_enter();
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const int o = owner[f], m = nb[f];
  if (o < 0 || o >= C || m < 0 || m >= C || o == m) {
    atomicOr(err, 1);
    return;
  }
  atomicAdd(&cnt[o], 1);
  atomicAdd(&cnt[m], 1);
}

__global__ void k_fill_ones(int32_t* __restrict__ a, int n) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = 1;
}

// Diagonal first in every row, then faces through a per-row cursor.
__global__ void k_place_diag(int C, const int32_t* __restrict__ rp, int32_t* __restrict__ col,
                             int32_t* __restrict__ src, int32_t* __restrict__ cursor) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C) return;
  col[rp[i]] = i;
  src[rp[i]] = -1 - i;
  cursor[i] = 1;
}

__global__ void k_place_faces(int F, const int32_t* __restrict__ owner, const int32_t* __restrict__ nb,
                              const int32_t* __restrict__ rp, int32_t* __restrict__ col,
                              int32_t* __restrict__ src, int32_t* __restrict__ cursor) {
  dep_enter();
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const int o = owner[f], m = nb[f];
  int p = rp[o] + atomicAdd(&cursor[o], 1);
  col[p] = m;
  src[p] = 2 * f;
  p = rp[m] + atomicAdd(&cursor[m], 1);
  col[p] = o;
  src[p] = 2 * f + 1;
}

// Thread per row: insertion sort by column (rows are short), duplicate check,
// and the LDU -> BSR position maps.
__global__ void k_sort_rows(int C, const int32_t* __restrict__ rp, int32_t* __restrict__ col,
                            int32_t* __restrict__ src, int32_t* __restrict__ pos_diag,
                            int32_t* __restrict__ pos_up, int32_t* __restrict__ pos_lo,
                            int32_t* __restrict__ err) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  // longest row -> err[2] (one atomic per warp)
  const int m = __reduce_max_sync(0xffffffffu, i < C ? rp[i + 1] - rp[i] : 0);
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(err + 2, m);
  if (i >= C) return;
  const int b = rp[i], e = rp[i + 1];
  for (int p = b + 1; p < e; ++p) {
    const int c = col[p], sv = src[p];
    int q = p - 1;
    while (q >= b && col[q] > c) {
      col[q + 1] = col[q];
      src[q + 1] = src[q];
      --q;
    }
    col[q + 1] = c;
    src[q + 1] = sv;
  }
  for (int p = b; p < e; ++p) {
    if (p > b && col[p] == col[p - 1]) atomicOr(err, 2);
    const int sv = src[p];
    if (sv < 0) pos_diag[-1 - sv] = p;
    else if (sv & 1) pos_lo[sv >> 1] = p;
    else pos_up[sv >> 1] = p;
  }
}

// Grid-stride over elements, GV_U independent elements per iteration (codes
// first, then values) so each thread keeps several loads in flight.
constexpr int GV_U = 4;

template <int NN>
__global__ void k_gather_values(size_t total, const int32_t* __restrict__ src,
                                const double* __restrict__ diag, const double* __restrict__ upper,
                                const double* __restrict__ lower, double* __restrict__ val) {
  dep_enter();
  const size_t S = (size_t)gridDim.x * blockDim.x;
  for (size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t0 < total; t0 += GV_U * S) {
    const double* a[GV_U];
#pragma unroll
    for (int u = 0; u < GV_U; ++u) {
      const size_t t = t0 + u * S;
      const size_t p = t < total ? t / NN : 0;
      const int e = (int)(t - p * NN);
      const int code = t < total ? __ldg(src + p) : -1;
      a[u] = (code < 0 ? diag + (size_t)(-1 - code) * NN : ((code & 1) ? lower : upper) + (size_t)(code >> 1) * NN) +
             (t < total ? e : 0);
    }
    double v[GV_U];
#pragma unroll
    for (int u = 0; u < GV_U; ++u) v[u] = t0 + u * S < total ? __ldg(a[u]) : 0.0;
#pragma unroll
    for (int u = 0; u < GV_U; ++u)
      if (t0 + u * S < total) val[t0 + u * S] = v[u];
  }
}

// The gather for a full setup, fused with the block Frobenius norms the
// first matching pass needs (N(M): fma sum of squares in row-major order
// from +0, then sqrt, as k_block_norms computes them), so the fine matrix is
// not read again for them. A warp takes 32 consecutive block-CSR positions:
// each source block (n*n contiguous doubles) is loaded by n*n lanes into a
// tile in shared memory (rows padded to an odd length: conflict-free), lane
// b then sums the squares of block b, and the tile is stored to the
// positions as one contiguous run. At a values-only resetup (nrm null) the
// kernel gathers without the norms and, given the fine level's slot map,
// lane b also stores block b into the fine level's thread-per-row copy.
constexpr int GN_U = 8;

template <int NN>
struct GnShape {
  static constexpr int NNP = NN | 1;          // padded tile row
  static constexpr int WARPS = NN <= 25 ? 4 : 2;
  static constexpr int LPB = NN < 32 ? NN : 32;  // lanes loading one block
};

// One block (n*n doubles, row-major, in shared memory) into its slot of the
// fine level's thread-per-row sliced copy (s32 or s16, the other null):
// slice lane slot % 32 of step tile slot / 32, each entry rounded to the
// cycle precision as k_tpr_fill rounds it (round to nearest).
template <int NN>
__device__ __forceinline__ void store_slot(const double* blk, int slot, float* s32, bf16* s16) {
  const int w = slot & 31;
  const size_t t = (size_t)(slot >> 5);
  if (s32) {
    using T = TprTile<NN, float>;
    float* tile = s32 + t * T::TILE;
#pragma unroll
    for (int g = 0; g < T::NG; ++g) {
      alignas(16) float v[T::G];
#pragma unroll
      for (int q = 0; q < T::G; ++q) v[q] = (float)blk[g * T::G + q];
      *reinterpret_cast<uint4*>(tile + g * T::G * 32 + w * T::G) = *reinterpret_cast<const uint4*>(v);
    }
#pragma unroll
    for (int r = 0; r < T::R; ++r) tile[T::NG * T::G * 32 + r * 32 + w] = (float)blk[T::NG * T::G + r];
  } else {
    using T = TprTile<NN, bf16>;
    bf16* tile = s16 + t * T::TILE;
#pragma unroll
    for (int g = 0; g < T::NG; ++g) {
      alignas(16) bf16 v[T::G];
#pragma unroll
      for (int q = 0; q < T::G; ++q) v[q] = __double2bfloat16(blk[g * T::G + q]);
      *reinterpret_cast<uint4*>(tile + g * T::G * 32 + w * T::G) = *reinterpret_cast<const uint4*>(v);
    }
#pragma unroll
    for (int r = 0; r < T::R; ++r) tile[T::NG * T::G * 32 + r * 32 + w] = __double2bfloat16(blk[T::NG * T::G + r]);
  }
}

template <int NN>
__global__ void __launch_bounds__(GnShape<NN>::WARPS * 32) k_gather_norms(int nnz, const int32_t* __restrict__ src,
                                                                         const double* __restrict__ diag,
                                                                         const double* __restrict__ upper,
                                                                         const double* __restrict__ lower,
                                                                         double* __restrict__ val,
                                                                         double* __restrict__ nrm,
                                                                         const int32_t* __restrict__ tpos,
                                                                         float* __restrict__ s32,
                                                                         bf16* __restrict__ s16) {
  dep_enter();
  using G = GnShape<NN>;
  __shared__ double tile[G::WARPS][32 * G::NNP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* tl = tile[warp];
  const int p0 = (blockIdx.x * G::WARPS + warp) * 32;
  if (p0 >= nnz) return;
  const int cnt = min(32, nnz - p0);
  const int code = lane < cnt ? __ldg(src + p0 + lane) : -1;
  const double* mine = code < 0 ? diag + (size_t)(-1 - code) * NN
                                : ((code & 1) ? lower : upper) + (size_t)(code >> 1) * NN;
  // GN_U source blocks in flight per lane (E entries of each)
  constexpr int E = (NN + 31) / 32;
  constexpr int U = GN_U / E > 0 ? GN_U / E : 1;
  for (int b0 = 0; b0 < cnt; b0 += U) {
    double v[U][E];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const double* a =
          reinterpret_cast<const double*>(__shfl_sync(0xffffffffu, (unsigned long long)mine, (b0 + u) & 31));
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int e = lane + 32 * j;
        v[u][j] = (b0 + u < cnt && e < NN) ? __ldg(a + e) : 0.0;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int e = lane + 32 * j;
        if (b0 + u < cnt && e < NN) tl[(b0 + u) * G::NNP + e] = v[u][j];
      }
  }
  __syncwarp();
  if (lane < cnt) {
    if (nrm) {
      double acc = 0.0;
#pragma unroll
      for (int e = 0; e < NN; ++e) {
        const double v = tl[lane * G::NNP + e];
        acc = fma(v, v, acc);
      }
      nrm[p0 + lane] = sqrt(acc);
    }
    if (tpos) store_slot<NN>(tl + lane * G::NNP, __ldg(tpos + p0 + lane), s32, s16);
  }
  double* out = val + (size_t)p0 * NN;
  for (int q = lane; q < cnt * NN; q += 32) out[q] = tl[(q / NN) * G::NNP + q % NN];
}

// Scatter of consecutive LDU blocks (one array: diag, upper or lower) to
// their block-CSR positions, with their Frobenius norms when nrm is given:
// a warp loads 32 contiguous source blocks into a tile (coalesced), lane b
// sums the squares of block b as k_block_norms does, and each block is
// stored whole at its position.
template <int NN>
__global__ void __launch_bounds__(GnShape<NN>::WARPS * 32) k_scatter_blocks(int count, const double* __restrict__ src,
                                                                           const int32_t* __restrict__ pos,
                                                                           double* __restrict__ val,
                                                                           double* __restrict__ nrm,
                                                                           const int32_t* __restrict__ tpos,
                                                                           float* __restrict__ s32,
                                                                           bf16* __restrict__ s16) {
  dep_enter();
  using G = GnShape<NN>;
  __shared__ double tile[G::WARPS][32 * G::NNP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* tl = tile[warp];
  const int b0 = (blockIdx.x * G::WARPS + warp) * 32;
  if (b0 >= count) return;
  const int cnt = min(32, count - b0);
  const double* in = src + (size_t)b0 * NN;
  for (int q = lane; q < cnt * NN; q += 32) tl[(q / NN) * G::NNP + q % NN] = __ldg(in + q);
  const int my = lane < cnt ? __ldg(pos + b0 + lane) : 0;
  __syncwarp();
  if (lane < cnt) {
    if (nrm) {
      double acc = 0.0;
#pragma unroll
      for (int e = 0; e < NN; ++e) {
        const double v = tl[lane * G::NNP + e];
        acc = fma(v, v, acc);
      }
      nrm[my] = sqrt(acc);
    }
    if (tpos) store_slot<NN>(tl + lane * G::NNP, __ldg(tpos + my), s32, s16);
  }
  for (int b = 0; b < cnt; ++b) {
    const int p = __shfl_sync(0xffffffffu, my, b);
    for (int e = lane; e < NN; e += 32) val[(size_t)p * NN + e] = tl[b * G::NNP + e];
  }
}

}  // namespace

bcs_status build_structure(Solver* s, const int32_t* owner, const int32_t* nb) {
  const int C = s->C, F = s->F;
  const size_t nnz = (size_t)C + 2 * (size_t)F;
  // block counts are int32 throughout; element offsets are computed in 64
  // bits, but keep every value array's element count in int32 range too
  if (nnz * (size_t)s->n * s->n > (size_t)INT32_MAX)
    return s->fail(BCS_EINVAL, "too many blocks for int32 indexing");
  s->nnz = (int)nnz;
  s->lv.clear();
  s->lv.emplace_back();
  Bsr& A = s->lv[0].A;
  A.rows = A.cols = C;
  A.nnz = (int)nnz;
  DBuf<int32_t> cnt, cursor;
  BCS_ALLOC(s, cnt, C);
  BCS_ALLOC(s, cursor, C);
  BCS_ALLOC(s, A.rp, C + 1);
  BCS_ALLOC(s, A.ci, nnz);
  BCS_ALLOC(s, s->src, nnz);
  BCS_ALLOC(s, s->pos_diag, C);
  BCS_ALLOC(s, s->pos_up, F > 0 ? F : 1);
  BCS_ALLOC(s, s->pos_lo, F > 0 ? F : 1);
  BCS_CU(s, cudaMemsetAsync(s->flag.p, 0, 4 * sizeof(int32_t), s->stream));
  BCS_LAUNCH_DEP(s, K_CONVERT, 4.0 * C, 0, k_fill_ones, grid_for(C, 256), 256, 0, cnt.p, C);
  if (F > 0)
    BCS_LAUNCH_DEP(s, K_CONVERT, 8.0 * F, 0, k_check_count, grid_for(F, 256), 256, 0, C, F, owner, nb, cnt.p,
               s->flag.p);
  // Reject bad ids before any kernel indexes rows with them.
  int32_t h = 0;
  BCS_CU(s, cudaMemcpyAsync(&h, s->flag.p, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  if (h & 1) return s->fail(BCS_EINVAL, "face addressing: cell id out of range or owner == neighbour");
  BCS_OKR(exclusive_scan(s, cnt.p, A.rp.p, C));
  BCS_LAUNCH_DEP(s, K_CONVERT, 12.0 * C, 0, k_place_diag, grid_for(C, 256), 256, 0, C, A.rp.p, A.ci.p, s->src.p,
             cursor.p);
  if (F > 0)
    BCS_LAUNCH_DEP(s, K_CONVERT, 24.0 * F, 0, k_place_faces, grid_for(F, 256), 256, 0, F, owner, nb, A.rp.p,
               A.ci.p, s->src.p, cursor.p);
  BCS_LAUNCH_DEP(s, K_CONVERT, 16.0 * nnz, 0, k_sort_rows, grid_for(C, 128), 128, 0, C, A.rp.p, A.ci.p,
             s->src.p, s->pos_diag.p, s->pos_up.p, s->pos_lo.p, s->flag.p);
  int32_t hf[3] = {0, 0, 0};
  BCS_CU(s, cudaMemcpyAsync(hf, s->flag.p, sizeof(hf), cudaMemcpyDeviceToHost, s->stream));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  if (hf[0] & 2) return s->fail(BCS_EINVAL, "face addressing: a face (cell pair) is repeated");
  A.maxrow = hf[2];
  return BCS_OK;
}

bcs_status permute_values(Solver* s, const double* diag, const double* upper, const double* lower) {
  Bsr& A = s->lv[0].A;
  const int n = s->n, nn = n * n;
  BCS_ALLOC(s, A.v, (size_t)A.nnz * nn);
  const size_t total = (size_t)A.nnz * nn;
  const double bytes = 16.0 * total + 4.0 * A.nnz;
  s->nrm0_fresh = false;
  s->v0_direct = -1;
  // the fine level's sliced copy written here too when its layout is known
  SliceTarget sl;
  BCS_OKR(fine_slice_target(s, &sl));
  const double slice_bytes = sl.tpos ? 4.0 * A.nnz + (double)total * (sl.s32 ? 4 : 2) : 0.0;
  const bool norms = !s->have_hierarchy;
  if (norms || sl.tpos) {
    // the tile gather: with the block norms when a full setup follows (its
    // first matching pass takes them), with the sliced copy when known
    if (norms) BCS_ALLOC(s, s->nrm0, A.nnz);
    BCS_OKR(with_n(n, [&](auto NC) -> bcs_status {
      constexpr int N = decltype(NC)::value;
      using G = GnShape<N * N>;
      BCS_LAUNCH_DEP(s, K_CONVERT, bytes + (norms ? 8.0 * A.nnz : 0.0) + slice_bytes, norms ? 2.0 * total : 0.0,
                 k_gather_norms<N * N>, grid_for((size_t)A.nnz, G::WARPS * 32), G::WARPS * 32, 0, A.nnz,
                 s->src.p, diag, upper, lower, A.v.p, norms ? s->nrm0.p : nullptr, sl.tpos, sl.s32, sl.s16);
      return BCS_OK;
    }));
    s->nrm0_fresh = norms;
    s->v0_direct = sl.prec;
    return BCS_OK;
  }
  return with_n(n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    unsigned grid = grid_for(total, 256);
    if (grid > 148u * 32u) grid = 148u * 32u;
    BCS_LAUNCH_DEP(s, K_CONVERT, bytes, 0, k_gather_values<N * N>, grid, 256, 0, total, s->src.p, diag, upper,
               lower, A.v.p);
    return BCS_OK;
  });
}

}  // namespace bcs

namespace bcs {

// Host values to the block-CSR values with the copy hidden behind the
// device work: the three LDU arrays go to the device in pieces on a second
// stream, and each piece is scattered (with its block norms when a full
// setup follows) as soon as it has landed.
bcs_status upload_values(Solver* s, const double* diag, const double* upper, const double* lower) {
  Bsr& A = s->lv[0].A;
  const int n = s->n, nn = n * n, C = s->C, F = s->F;
  BCS_ALLOC(s, A.v, (size_t)A.nnz * nn);
  BCS_ALLOC(s, s->stage_d, (size_t)C * nn);
  if (F > 0) {
    BCS_ALLOC(s, s->stage_u, (size_t)F * nn);
    BCS_ALLOC(s, s->stage_l, (size_t)F * nn);
  }
  const bool norms = !s->have_hierarchy;
  s->nrm0_fresh = false;
  s->v0_direct = -1;
  SliceTarget sl;
  BCS_OKR(fine_slice_target(s, &sl));
  if (norms) BCS_ALLOC(s, s->nrm0, A.nnz);
  if (!s->cstream) BCS_CU(s, cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking));
  struct Part {
    const double* host;
    double* dev;
    const int32_t* pos;
    int count;
  };
  const Part parts[3] = {{diag, s->stage_d.p, s->pos_diag.p, C},
                         {upper, s->stage_u.p, s->pos_up.p, F},
                         {lower, s->stage_l.p, s->pos_lo.p, F}};
  // pieces of about 64 MB
  const int piece = std::max(1, (int)((64u << 20) / ((size_t)nn * sizeof(double))));
  size_t ev = 0;
  auto next_event = [&](cudaEvent_t* e) -> bcs_status {
    if (ev == s->copy_events.size()) {
      cudaEvent_t x;
      BCS_CU(s, cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
      s->copy_events.push_back(x);
    }
    *e = s->copy_events[ev++];
    return BCS_OK;
  };
  // the copy stream starts after the allocations on the solver's stream
  cudaEvent_t e0;
  BCS_OKR(next_event(&e0));
  BCS_CU(s, cudaEventRecord(e0, s->stream));
  BCS_CU(s, cudaStreamWaitEvent(s->cstream, e0, 0));
  for (const Part& pt : parts) {
    for (int b = 0; b < pt.count; b += piece) {
      const int cnt = std::min(piece, pt.count - b);
      const size_t off = (size_t)b * nn;
      BCS_CU(s, cudaMemcpyAsync(pt.dev + off, pt.host + off, (size_t)cnt * nn * sizeof(double),
                                cudaMemcpyHostToDevice, s->cstream));
      cudaEvent_t e;
      BCS_OKR(next_event(&e));
      BCS_CU(s, cudaEventRecord(e, s->cstream));
      BCS_CU(s, cudaStreamWaitEvent(s->stream, e, 0));
      BCS_OKR(with_n(n, [&](auto NC) -> bcs_status {
        constexpr int N = decltype(NC)::value;
        using G = GnShape<N * N>;
        BCS_LAUNCH_DEP(s, K_CONVERT,
                   16.0 * cnt * N * N + 4.0 * cnt + (norms ? 8.0 * cnt : 0.0) +
                       (sl.tpos ? 4.0 * cnt + (double)cnt * N * N * (sl.s32 ? 4 : 2) : 0.0),
                   norms ? 2.0 * cnt * N * N : 0.0, k_scatter_blocks<N * N>, grid_for(cnt, G::WARPS * 32),
                   G::WARPS * 32, 0, cnt, pt.dev + off, pt.pos + b, A.v.p, norms ? s->nrm0.p : nullptr, sl.tpos,
                   sl.s32, sl.s16);
        return BCS_OK;
      }));
    }
  }
  s->nrm0_fresh = norms;
  s->v0_direct = sl.prec;
  return BCS_OK;
}

}  // namespace bcs
