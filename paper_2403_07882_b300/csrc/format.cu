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
#include "internal.h"

namespace bcs {

namespace {

__global__ void k_check_count(int C, int F, const int32_t* __restrict__ owner,
                              const int32_t* __restrict__ nb, int32_t* __restrict__ cnt,
                              int32_t* __restrict__ err) {
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
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = 1;
}

// Diagonal first in every row, then faces through a per-row cursor.
__global__ void k_place_diag(int C, const int32_t* __restrict__ rp, int32_t* __restrict__ col,
                             int32_t* __restrict__ src, int32_t* __restrict__ cursor) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C) return;
  col[rp[i]] = i;
  src[rp[i]] = -1 - i;
  cursor[i] = 1;
}

__global__ void k_place_faces(int F, const int32_t* __restrict__ owner, const int32_t* __restrict__ nb,
                              const int32_t* __restrict__ rp, int32_t* __restrict__ col,
                              int32_t* __restrict__ src, int32_t* __restrict__ cursor) {
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
  BCS_LAUNCH(s, K_CONVERT, 4.0 * C, 0, k_fill_ones, grid_for(C, 256), 256, 0, cnt.p, C);
  if (F > 0)
    BCS_LAUNCH(s, K_CONVERT, 8.0 * F, 0, k_check_count, grid_for(F, 256), 256, 0, C, F, owner, nb, cnt.p,
               s->flag.p);
  // Reject bad ids before any kernel indexes rows with them.
  int32_t h = 0;
  BCS_CU(s, cudaMemcpyAsync(&h, s->flag.p, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  if (h & 1) return s->fail(BCS_EINVAL, "face addressing: cell id out of range or owner == neighbour");
  BCS_OKR(exclusive_scan(s, cnt.p, A.rp.p, C));
  BCS_LAUNCH(s, K_CONVERT, 12.0 * C, 0, k_place_diag, grid_for(C, 256), 256, 0, C, A.rp.p, A.ci.p, s->src.p,
             cursor.p);
  if (F > 0)
    BCS_LAUNCH(s, K_CONVERT, 24.0 * F, 0, k_place_faces, grid_for(F, 256), 256, 0, F, owner, nb, A.rp.p,
               A.ci.p, s->src.p, cursor.p);
  BCS_LAUNCH(s, K_CONVERT, 16.0 * nnz, 0, k_sort_rows, grid_for(C, 128), 128, 0, C, A.rp.p, A.ci.p,
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
  return with_n(n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    unsigned grid = grid_for(total, 256);
    if (grid > 148u * 32u) grid = 148u * 32u;
    BCS_LAUNCH(s, K_CONVERT, bytes, 0, k_gather_values<N * N>, grid, 256, 0, total, s->src.p, diag, upper,
               lower, A.v.p);
    return BCS_OK;
  });
}

}  // namespace bcs
