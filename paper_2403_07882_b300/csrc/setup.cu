// Aggregation AMG setup for block-coupled systems (Sec. 2.3: aggregation
// AMG built by graph matching; block smoothers). All setup arithmetic is FP64
// and every value is produced by one thread in a fixed operation order with
// explicit fma, so the hierarchy is identical bit for bit across runs and
// equal to the CPU reference's.
//
// Reading of the unstated rules (the paper names graph matching only):
//  * strength: w_ij = (N(A_ij) + N(A_ji)) / (2 max(N(A_ii), N(A_jj))),
//    N = Frobenius norm (fma sum of squares in row-major order, then sqrt);
//  * synchronous handshake matching rounds: each unmatched row picks the
//    unmatched neighbour of largest positive weight (smaller index on ties),
//    mutual picks pair up;
//  * unmatched rows join the aggregate of their strongest matched neighbour,
//    if any; aggregates are numbered by ascending smallest member;
//  * a second pass repeats this on the aggregate graph (block sums), giving
//    aggregates of about four rows;
//  * Galerkin coarse operator R A P with R = P^T; P tentative (identity
//    blocks, the default) or smoothed (I - omega_P D^-1 A) P_tent with
//    omega_P = p_omega / max_i sum_j ||D_i^-1 A_ij||_inf;
//  * block inverses by Gauss-Jordan with implicit partial pivoting;
//  * coarsest level: dense Gauss-Jordan inverse (FP64), applied as a GEMV.
#include <cooperative_groups.h>

#include <climits>
#include <utility>

#include "internal.h"
#include "gj.cuh"

namespace cg = cooperative_groups;

namespace bcs {

namespace {

__device__ __forceinline__ int find_col(const int32_t* __restrict__ ci, int b, int e, int j) {
  while (b < e) {
    const int m = (b + e) >> 1;
    const int c = ci[m];
    if (c == j) return m;
    if (c < j) b = m + 1;
    else e = m;
  }
  return -1;
}

__global__ void k_diag_pos(int rows, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           int32_t* __restrict__ dpos, int32_t* __restrict__ err) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const int p = find_col(ci, rp[i], rp[i + 1], i);
  dpos[i] = p;
  if (p < 0) atomicOr(err, 4);
}

// The FP32 / BF16 block-Jacobi cycle's inverses computed in FP32 (the FP32
// pipe is many times the FP64 one): each diagonal block rounded to FP32 and
// inverted by the same Gauss-Jordan in FP32 arithmetic.
template <int N>
__global__ void __launch_bounds__(64) k_block_inverse32(int rows, const int32_t* __restrict__ dpos,
                                                        const double* __restrict__ val, float* __restrict__ dinv,
                                                        int32_t* __restrict__ err) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const int dp = dpos[i];
  if (dp < 0) return;
  BlockGJ<N, float> g;
  const double* a = val + (size_t)dp * N * N;
#pragma unroll
  for (int r = 0; r < N; ++r)
#pragma unroll
    for (int c = 0; c < N; ++c) g.M[r][c] = (float)a[r * N + c];
  if (!gj_finish<N>(g, dinv + (size_t)i * N * N)) atomicOr(err, 8);
}

template <int N>
__global__ void __launch_bounds__(64) k_block_inverse(int rows, const int32_t* __restrict__ dpos,
                                                      const double* __restrict__ val, double* __restrict__ dinv,
                                                      int32_t* __restrict__ err) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const int dp = dpos[i];
  if (dp < 0) return;
  BlockGJ<N> g;
  const double* a = val + (size_t)dp * N * N;
#pragma unroll
  for (int r = 0; r < N; ++r)
#pragma unroll
    for (int c = 0; c < N; ++c) g.M[r][c] = a[r * N + c];
  if (!gj_finish<N>(g, dinv + (size_t)i * N * N)) atomicOr(err, 8);
}

template <int NN>
__global__ void k_block_norms(int nnz, const double* __restrict__ val, double* __restrict__ nrm) {
  dep_enter();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  const double* a = val + (size_t)k * NN;
  double acc = 0.0;
#pragma unroll
  for (int e = 0; e < NN; ++e) acc = fma(a[e], a[e], acc);
  nrm[k] = sqrt(acc);
}

__global__ void k_row_index(int rows, const int32_t* __restrict__ rp, int32_t* __restrict__ ridx) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  for (int k = rp[i]; k < rp[i + 1]; ++k) ridx[k] = i;
}

__global__ void k_weights(int nnz, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const int32_t* __restrict__ ridx, const int32_t* __restrict__ dpos,
                          const double* __restrict__ nrm, double* __restrict__ w) {
  dep_enter();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  const int i = ridx[k], j = ci[k];
  if (i == j) {
    w[k] = 0.0;
    return;
  }
  const int kt = find_col(ci, rp[j], rp[j + 1], i);
  const double s = nrm[k] + (kt >= 0 ? nrm[kt] : 0.0);
  const double di = dpos[i] >= 0 ? nrm[dpos[i]] : 0.0;
  const double dj = dpos[j] >= 0 ? nrm[dpos[j]] : 0.0;
  const double d = 2.0 * (di < dj ? dj : di);
  w[k] = d > 0.0 ? s / d : 0.0;
}

__global__ void k_choose(int rows, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const double* __restrict__ w, const int32_t* __restrict__ mate,
                         int32_t* __restrict__ choice) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  int best = -1;
  if (mate[i] < 0) {
    double bw = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      const int j = ci[k];
      if (j == i || mate[j] >= 0) continue;
      if (w[k] > bw) {
        bw = w[k];
        best = j;
      }
    }
  }
  choice[i] = best;
}

__global__ void k_pair(int rows, const int32_t* __restrict__ choice, int32_t* __restrict__ mate) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const int c = choice[i];
  if (mate[i] < 0 && c >= 0 && choice[c] == i) mate[i] = c;
}

__global__ void k_root(int rows, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                       const double* __restrict__ w, const int32_t* __restrict__ mate,
                       int32_t* __restrict__ root, int32_t* __restrict__ amin) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  int r;
  if (mate[i] >= 0) {
    r = min(i, mate[i]);
  } else {
    int best = -1;
    double bw = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      const int j = ci[k];
      if (j == i || mate[j] < 0) continue;
      if (w[k] > bw) {
        bw = w[k];
        best = j;
      }
    }
    r = best >= 0 ? min(best, mate[best]) : i;
  }
  root[i] = r;
  atomicMin(&amin[r], i);
}

__global__ void k_is_min(int rows, const int32_t* __restrict__ root, const int32_t* __restrict__ amin,
                         int32_t* __restrict__ flag) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < rows) flag[i] = amin[root[i]] == i ? 1 : 0;
}

__global__ void k_assign(int rows, const int32_t* __restrict__ root, const int32_t* __restrict__ amin,
                         const int32_t* __restrict__ id, int32_t* __restrict__ agg) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < rows) agg[i] = id[amin[root[i]]];
}

__global__ void k_compose(int rows, const int32_t* __restrict__ a2, int32_t* __restrict__ agg) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < rows) agg[i] = a2[agg[i]];
}

__global__ void k_fill_int(int32_t* __restrict__ a, int n, int v) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

__global__ void k_count_by(int m, const int32_t* __restrict__ key, int32_t* __restrict__ cnt) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) atomicAdd(&cnt[key[i]], 1);
}

// out[ptr[key[q]] + slot] = val ? val[q] : q
__global__ void k_place_by(int m, const int32_t* __restrict__ key, const int32_t* __restrict__ val,
                           const int32_t* __restrict__ ptr, int32_t* __restrict__ cursor,
                           int32_t* __restrict__ out) {
  dep_enter();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < m) out[ptr[key[q]] + atomicAdd(&cursor[key[q]], 1)] = val ? val[q] : q;
}

// Block-reduced maximum: one atomic per block (an atomic per element on one
// address serialises millions of updates).
__global__ void k_max_int(int n, const int32_t* __restrict__ a, int32_t* __restrict__ out) {
  dep_enter();
  __shared__ int32_t wm[32];
  int v = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v = max(v, a[i]);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, d));
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, wm[w]);
    atomicMax(out, m);
  }
}

__global__ void k_compact(int rows, const int32_t* __restrict__ cptr, const int32_t* __restrict__ cand,
                          const int32_t* __restrict__ rp, int32_t* __restrict__ ci) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const int b = cptr[i], o = rp[i], len = rp[i + 1] - rp[i];
  for (int q = 0; q < len; ++q) ci[o + q] = cand[b + q];
}

// Tentative Galerkin pattern and gather lists from one segmented sort. A
// candidate packs (coarse column agg(j)) << 32 | (fine block position); the
// candidates of coarse row I are the blocks of its member rows, sorted
// ascending, so each run of equal column is one coarse block and lists its
// fine blocks in ascending position (members ascending, columns ascending
// within a row), the summation order of the definition.

// Candidate count of coarse row I (its members' row lengths); longest -> *mx;
// moff[i] = where member row i's candidates start inside its coarse row.
__global__ void k_cand_count_tent(int nagg, const int32_t* __restrict__ mptr, const int32_t* __restrict__ mem,
                                  const int32_t* __restrict__ rp, int32_t* __restrict__ cnt, int32_t* __restrict__ moff,
                                  int32_t* __restrict__ mx) {
  dep_enter();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  int c = 0;
  if (I < nagg)
    for (int q = mptr[I]; q < mptr[I + 1]; ++q) {
      const int i = mem[q];
      moff[i] = c;
      c += rp[i + 1] - rp[i];
    }
  const int m = __reduce_max_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(mx, m);
  if (I < nagg) cnt[I] = c;
}

// One thread per fine row: its blocks' candidates (coarse column agg(j),
// fine block position p), contiguous in its coarse row's segment. Sorting a
// segment by (column, position) groups each coarse block's fine blocks in
// ascending position, the summation order of the definition.
__global__ void k_cand_pack_tent(int rows, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                 const int32_t* __restrict__ agg, const int32_t* __restrict__ cptr,
                                 const int32_t* __restrict__ moff, uint64_t* __restrict__ cand) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const long long o = (long long)cptr[agg[i]] + moff[i] - rp[i];
  for (int p = rp[i]; p < rp[i + 1]; ++p) cand[o + p] = ((uint64_t)(uint32_t)agg[ci[p]] << 32) | (uint32_t)p;
}

// Runs (distinct columns) of the sorted segments, one warp per segment: lane
// l looks at candidate t0 + l of each 32-candidate chunk; a candidate starts
// a run when it is the segment's first or its column differs from the one
// before it.
struct RunScan {
  unsigned first_mask;
  uint32_t J;
  bool live, first;
};

__device__ __forceinline__ RunScan run_chunk(const uint64_t* __restrict__ cand, int t, int t0, int t1,
                                             uint32_t* carry) {
  const int lane = threadIdx.x & 31;
  RunScan r;
  r.live = t < t1;
  r.J = r.live ? (uint32_t)(__ldg(cand + t) >> 32) : 0u;
  uint32_t prev = __shfl_up_sync(0xffffffffu, r.J, 1);
  if (lane == 0) prev = *carry;
  r.first = r.live && (t == t0 || r.J != prev);
  r.first_mask = __ballot_sync(0xffffffffu, r.first);
  *carry = __shfl_sync(0xffffffffu, r.J, 31);
  return r;
}

// Number of runs of each segment; the longest -> *mx when mx is given (one
// atomic per block: warps loop over the segments, the block reduces).
constexpr int RC_BLOCKS = 148 * 8;

__global__ void __launch_bounds__(256) k_runs_count(int rows, const int32_t* __restrict__ seg,
                                                    const uint64_t* __restrict__ cand, int32_t* __restrict__ cnt,
                                                    int32_t* __restrict__ mx) {
  dep_enter();
  __shared__ int wm[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int best = 0;
  for (int I = blockIdx.x * 8 + warp; I < rows; I += gridDim.x * 8) {
    const int t0 = seg[I], t1 = seg[I + 1];
    uint32_t carry = 0;
    int c = 0;
    for (int b = t0; b < t1; b += 32) {
      const RunScan r = run_chunk(cand, b + lane, t0, t1, &carry);
      c += __popc(r.first_mask);
    }
    if (lane == 0) cnt[I] = c;
    best = max(best, c);
  }
  if (lane == 0) wm[warp] = best;
  __syncthreads();
  if (threadIdx.x == 0 && mx) {
    int m = 0;
    for (int w = 0; w < 8; ++w) m = max(m, wm[w]);
    if (m > 0) atomicMax(mx, m);
  }
}

// One output block per run: column col[o]. The sorted candidates are also
// the plan of the value sum: sk[t] = fine block position, with the sign bit
// set on the first candidate of each run.
constexpr int32_t TS_FIRST = INT32_MIN;

__global__ void k_runs_emit(int rows, const int32_t* __restrict__ seg, const uint64_t* __restrict__ cand,
                            const int32_t* __restrict__ rp, int32_t* __restrict__ col, int32_t* __restrict__ sk) {
  dep_enter();
  const int I = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (I >= rows) return;
  const int lane = threadIdx.x & 31;
  const int t0 = seg[I], t1 = seg[I + 1];
  uint32_t carry = 0;
  int o = rp[I] - 1;
  for (int b = t0; b < t1; b += 32) {
    const int t = b + lane;
    const RunScan r = run_chunk(cand, t, t0, t1, &carry);
    const int mine = o + __popc(r.first_mask & (0xffffffffu >> (31 - lane)));
    if (r.first) col[mine] = (int32_t)r.J;
    if (r.live) {
      const int32_t p = (int32_t)(uint32_t)__ldg(cand + t);
      sk[t] = r.first ? (p | TS_FIRST) : p;
    }
    o += __popc(r.first_mask);
  }
}

__device__ __forceinline__ double plus_zero(double v) {
  const long long b = __double_as_longlong(v);
  return b == (long long)0x8000000000000000ll ? 0.0 : v;  // 0 + v, without the add
}

// Coarse block values of P_tent^T A P_tent: out[q] = left-to-right FP64 sum
// from +0 of the fine blocks of q in position order. The plan lists each
// coarse row's terms sorted by (output block, fine position), so the terms
// of every output are consecutive and in position order: one group of lanes
// per coarse row walks them with its running sums in registers and stores a
// sum when the next output starts. Lane e of a group owns entry e (and
// e + 32, ... when n^2 > 32) of every block. The first term of an output is
// stored, not added: 0 + v equals v except that -0 becomes +0 (integer
// operations), so no FP64 add is spent on it. TS_U fine blocks are fetched
// per round trip, their positions one round ahead.
constexpr int TS_U = 8;
constexpr int TS_WARPS = 4;

template <int NN>
struct TentShape {
  static constexpr int W = NN >= 32 ? 32 : NN;  // lanes per coarse row
  static constexpr int G = 32 / W;              // coarse rows per warp
  static constexpr int E = (NN + 31) / 32;      // entries per lane
};

template <int NN>
__global__ void __launch_bounds__(TS_WARPS * 32) k_tent_sum(int nagg, const int32_t* __restrict__ seg,
                                                           const int32_t* __restrict__ sk,
                                                           const int32_t* __restrict__ crp,
                                                           const double* __restrict__ src, double* __restrict__ out) {
  dep_enter();
  using S = TentShape<NN>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / S::W, e0 = lane - g * S::W;
  const int I = (blockIdx.x * TS_WARPS + warp) * S::G + g;
  if (g >= S::G || I >= nagg) return;
  const int t0 = seg[I], t1 = seg[I + 1];
  const int obase = crp[I];
  int o = obase - 1;
  double acc[S::E];
#pragma unroll
  for (int j = 0; j < S::E; ++j) acc[j] = 0.0;
  int kn[TS_U];
#pragma unroll
  for (int u = 0; u < TS_U; ++u) kn[u] = t0 + u < t1 ? __ldg(sk + t0 + u) : 0;
  for (int t = t0; t < t1; t += TS_U) {
    int k[TS_U];
#pragma unroll
    for (int u = 0; u < TS_U; ++u) k[u] = kn[u];
    double v[TS_U][S::E];
#pragma unroll
    for (int u = 0; u < TS_U; ++u)
#pragma unroll
      for (int j = 0; j < S::E; ++j) {
        const int e = e0 + j * S::W;
        v[u][j] = (t + u < t1 && e < NN) ? __ldg(src + (size_t)(k[u] & INT32_MAX) * NN + e) : 0.0;
      }
#pragma unroll
    for (int u = 0; u < TS_U; ++u) kn[u] = t + TS_U + u < t1 ? __ldg(sk + t + TS_U + u) : 0;
#pragma unroll
    for (int u = 0; u < TS_U; ++u) {
      if (t + u >= t1) break;
      if (k[u] < 0) {
        if (o >= obase)
#pragma unroll
          for (int j = 0; j < S::E; ++j)
            if (e0 + j * S::W < NN) out[(size_t)o * NN + e0 + j * S::W] = acc[j];
        ++o;
#pragma unroll
        for (int j = 0; j < S::E; ++j) acc[j] = plus_zero(v[u][j]);
      } else {
#pragma unroll
        for (int j = 0; j < S::E; ++j) acc[j] = acc[j] + v[u][j];
      }
    }
  }
  if (o >= obase)
#pragma unroll
    for (int j = 0; j < S::E; ++j)
      if (e0 + j * S::W < NN) out[(size_t)o * NN + e0 + j * S::W] = acc[j];
}

// ----------------------------------------------------- smoothed prolongation
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

template <int N>
__global__ void k_rho(int rows, const int32_t* __restrict__ rp, const double* __restrict__ val,
                      const double* __restrict__ dinv, double* __restrict__ rho) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const double* D = dinv + (size_t)i * N * N;
  double s = 0.0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    const double* a = val + (size_t)k * N * N;
    double mx = 0.0;
    for (int r = 0; r < N; ++r) {
      double rs = 0.0;
      for (int c = 0; c < N; ++c) {
        double t = 0.0;
        for (int m = 0; m < N; ++m) t = fma(D[r * N + m], a[m * N + c], t);
        rs = rs + fabs(t);
      }
      if (rs > mx) mx = rs;
    }
    s = s + mx;
  }
  atomic_max_nonneg(rho, s);
}

__global__ void k_cand_count_p(int rows, const int32_t* __restrict__ rp, int32_t* __restrict__ cnt) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < rows) cnt[i] = rp[i + 1] - rp[i];
}

__global__ void k_cand_fill_p(int rows, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const int32_t* __restrict__ agg, int32_t* __restrict__ cand) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  for (int k = rp[i]; k < rp[i + 1]; ++k) cand[k] = agg[ci[k]];
}

// P block (i, J) = fma(-omega, D_i^-1 S_iJ, delta), S_iJ = sum (row order) of
// A_ik over neighbours k in aggregate J.
template <int N>
__global__ void k_p_values(int pnnz, const int32_t* __restrict__ prow, const int32_t* __restrict__ pci,
                           const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ val, const double* __restrict__ dinv,
                           const int32_t* __restrict__ agg, double omega, double* __restrict__ pv) {
  dep_enter();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= pnnz) return;
  const int i = prow[q], J = pci[q];
  double S[N * N];
#pragma unroll
  for (int e = 0; e < N * N; ++e) S[e] = 0.0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    if (agg[ci[k]] != J) continue;
    const double* a = val + (size_t)k * N * N;
#pragma unroll
    for (int e = 0; e < N * N; ++e) S[e] = S[e] + a[e];
  }
  const double* D = dinv + (size_t)i * N * N;
  const bool own = agg[i] == J;
  double* o = pv + (size_t)q * N * N;
  for (int r = 0; r < N; ++r)
    for (int c = 0; c < N; ++c) {
      double t = 0.0;
#pragma unroll
      for (int m = 0; m < N; ++m) t = fma(D[r * N + m], S[m * N + c], t);
      o[r * N + c] = fma(-omega, t, (own && r == c) ? 1.0 : 0.0);
    }
}

// R block (J, i) = P block (i, J)^T.
template <int N>
__global__ void k_transpose_values(int rnnz, const int32_t* __restrict__ rrow, const int32_t* __restrict__ rci,
                                   const int32_t* __restrict__ prp, const int32_t* __restrict__ pci,
                                   const double* __restrict__ pv, double* __restrict__ rv) {
  dep_enter();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= rnnz) return;
  const int J = rrow[q], i = rci[q];
  const int kk = find_col(pci, prp[i], prp[i + 1], J);
  const double* a = pv + (size_t)kk * N * N;
  double* o = rv + (size_t)q * N * N;
  for (int r = 0; r < N; ++r)
    for (int c = 0; c < N; ++c) o[r * N + c] = a[c * N + r];
}

// General block SpGEMM C = A B.
__global__ void k_cand_count_gemm(int rows, const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
                                  const int32_t* __restrict__ brp, int32_t* __restrict__ cnt) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  int c = 0;
  for (int k = arp[i]; k < arp[i + 1]; ++k) c += brp[aci[k] + 1] - brp[aci[k]];
  cnt[i] = c;
}

__global__ void k_cand_fill_gemm(int rows, const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
                                 const int32_t* __restrict__ brp, const int32_t* __restrict__ bci,
                                 const int32_t* __restrict__ cptr, int32_t* __restrict__ cand) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  int o = cptr[i];
  for (int k = arp[i]; k < arp[i + 1]; ++k) {
    const int j = aci[k];
    for (int kk = brp[j]; kk < brp[j + 1]; ++kk) cand[o++] = bci[kk];
  }
}

// C_iJ[r][c] = over k of A's row i (ascending), then m ascending,
// fma(A_ik[r][m], B_kJ[m][c], acc), from +0.
template <int N>
__global__ void k_gemm_values(int cnnz, const int32_t* __restrict__ crow, const int32_t* __restrict__ cci,
                              const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
                              const double* __restrict__ av, const int32_t* __restrict__ brp,
                              const int32_t* __restrict__ bci, const double* __restrict__ bv,
                              double* __restrict__ cv) {
  dep_enter();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= cnnz) return;
  const int i = crow[q], J = cci[q];
  double acc[N * N];
#pragma unroll
  for (int e = 0; e < N * N; ++e) acc[e] = 0.0;
  for (int k = arp[i]; k < arp[i + 1]; ++k) {
    const int j = aci[k];
    const int kk = find_col(bci, brp[j], brp[j + 1], J);
    if (kk < 0) continue;
    const double* a = av + (size_t)k * N * N;
    const double* b = bv + (size_t)kk * N * N;
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
      for (int c = 0; c < N; ++c)
#pragma unroll
        for (int m = 0; m < N; ++m) acc[r * N + c] = fma(a[r * N + m], b[m * N + c], acc[r * N + c]);
  }
  double* o = cv + (size_t)q * N * N;
#pragma unroll
  for (int e = 0; e < N * N; ++e) o[e] = acc[e];
}

// ------------------------------------------------------------ coarse inverse
__global__ void k_dense_from_bsr(int rows, int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                 const double* __restrict__ val, double* __restrict__ M, int N) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const size_t W = 2 * (size_t)N;
  for (int r = 0; r < n; ++r) {
    double* row = M + (size_t)(i * n + r) * W;
    for (size_t j = 0; j < W; ++j) row[j] = 0.0;
    row[N + i * n + r] = 1.0;
  }
  for (int k = rp[i]; k < rp[i + 1]; ++k)
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c)
        M[(size_t)(i * n + r) * W + ci[k] * n + c] = val[(size_t)k * n * n + r * n + c];
}

// Gauss-Jordan on [A | I] (N x 2N) over a cooperative grid, one grid barrier
// per pivot step. Step k: every block finds the same pivot among the unused
// rows from colbuf[k & 1] (column k as it stood after step k-1); each block
// updates its own rows i != p for columns j >= k and records their column
// k+1 in colbuf[(k + 1) & 1]; the pivot row is only read in step k.
__global__ void k_gauss_jordan(int N, double* __restrict__ M, double* __restrict__ colbuf,
                               int32_t* __restrict__ prow_out, int32_t* __restrict__ err) {
  dep_enter();
  cg::grid_group grid = cg::this_grid();
  extern __shared__ unsigned char used[];  // N flags
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_p;
  __shared__ double s_l;
  const size_t W = 2 * (size_t)N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) used[i] = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    colbuf[i] = M[(size_t)i * W];
  grid.sync();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < N; ++k) {
    const double* col = colbuf + (size_t)(k & 1) * N;
    double bv = -1.0;
    int bi = INT_MAX;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      if (used[i]) continue;
      const double v = fabs(col[i]);
      if (v > bv || (v == bv && i < bi)) {
        bv = v;
        bi = i;
      }
    }
    for (int d = 16; d > 0; d >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, bv, d);
      const int oi = __shfl_down_sync(0xffffffffu, bi, d);
      if (ov > bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      red_v[warp] = bv;
      red_i[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = red_v[0];
      int p = red_i[0];
      for (int w = 1; w < nw; ++w)
        if (red_v[w] > v || (red_v[w] == v && red_i[w] < p)) {
          v = red_v[w];
          p = red_i[w];
        }
      s_p = p;
      if (p != INT_MAX) {
        used[p] = 1;
        if (blockIdx.x == 0) prow_out[k] = p;
      }
    }
    __syncthreads();
    const int p = s_p;
    // no pivot candidate (a column of NaNs) or a zero pivot: singular
    const double piv = p == INT_MAX ? 0.0 : M[(size_t)p * W + k];
    const double* prow = M + (size_t)(p == INT_MAX ? 0 : p) * W;
    if (piv == 0.0) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, 16);
      return;  // every block sees the same pivot and leaves before the next barrier
    }
    const double rpiv = 1.0 / piv;
    double* nxt = colbuf + (size_t)((k + 1) & 1) * N;
    for (int i = blockIdx.x; i < N; i += gridDim.x) {
      if (i == p) {
        if (threadIdx.x == 0 && k + 1 < N) nxt[i] = prow[k + 1];
        continue;
      }
      double* row = M + (size_t)i * W;
      if (threadIdx.x == 0) s_l = row[k] * rpiv;
      __syncthreads();
      const double l = s_l;
      for (size_t j = k + threadIdx.x; j < W; j += blockDim.x) row[j] = fma(-l, prow[j], row[j]);
      __syncthreads();
      if (threadIdx.x == 0 && k + 1 < N) nxt[i] = row[k + 1];
    }
    grid.sync();
  }
}

// The same Gauss-Jordan for small N on one block with [A | I] in shared
// memory: the same pivot choice and the same operation on every element as
// k_gauss_jordan (one warp per row, the block's barrier per pivot step);
// the reduced [A | I] and the pivot rows are written back for k_gj_finish.
constexpr int GJ_SMEM_THREADS = 512;

__global__ void __launch_bounds__(GJ_SMEM_THREADS) k_gauss_jordan_smem(int N, double* __restrict__ M,
                                                                       int32_t* __restrict__ prow_out,
                                                                       int32_t* __restrict__ err) {
  dep_enter();
  extern __shared__ double sm[];  // N x 2N, then N used flags
  unsigned char* used = reinterpret_cast<unsigned char*>(sm + 2 * (size_t)N * N);
  __shared__ int s_p;
  __shared__ double s_rpiv;
  const int W = 2 * N;
  for (int t = threadIdx.x; t < N * W; t += blockDim.x) sm[t] = M[t];
  for (int i = threadIdx.x; i < N; i += blockDim.x) used[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < N; ++k) {
    if (warp == 0) {
      // largest |M[i][k]| over the unused rows, the lowest i on ties: the
      // bit patterns of non-negative doubles order like their values, so
      // integer compares pick the same row as floating-point ones (NaN,
      // which no floating-point compare picks, is skipped)
      long long bk = -1;
      int bi = INT_MAX;
      for (int i = lane; i < N; i += 32) {
        const double v = sm[i * W + k];
        if (used[i] || isnan(v)) continue;
        const long long key = __double_as_longlong(v) & 0x7fffffffffffffffll;
        if (key > bk || (key == bk && i < bi)) {
          bk = key;
          bi = i;
        }
      }
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        const long long ok = __shfl_down_sync(0xffffffffu, bk, d);
        const int oi = __shfl_down_sync(0xffffffffu, bi, d);
        if (ok > bk || (ok == bk && oi < bi)) {
          bk = ok;
          bi = oi;
        }
      }
      if (lane == 0) {
        s_p = bi;
        if (bi != INT_MAX) {
          used[bi] = 1;
          prow_out[k] = bi;
          const double piv = sm[bi * W + k];
          s_rpiv = piv == 0.0 ? 0.0 : 1.0 / piv;
        }
      }
    }
    __syncthreads();
    const int p = s_p;
    if (p == INT_MAX || sm[p * W + k] == 0.0) {
      if (threadIdx.x == 0) atomicOr(err, 16);
      return;
    }
    const double* prow = sm + p * W;
    const double rpiv = s_rpiv;
    for (int i = warp; i < N; i += nw) {
      if (i == p) continue;
      double* row = sm + i * W;
      const double l = row[k] * rpiv;
      __syncwarp();  // every lane has read row[k] before lane 0 rewrites it
      for (int j = k + lane; j < W; j += 32) row[j] = fma(-l, prow[j], row[j]);
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < N * W; t += blockDim.x) M[t] = sm[t];
}

__global__ void k_gj_finish(int N, const double* __restrict__ M, const int32_t* __restrict__ prow,
                            double* __restrict__ inv) {
  dep_enter();
  const size_t W = 2 * (size_t)N;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)N * N;
       t += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(t / N), j = (int)(t % N);
    const int p = prow[k];
    inv[t] = M[(size_t)p * W + N + j] * (1.0 / M[(size_t)p * W + k]);
  }
}

}  // namespace

// ======================================================================= host
namespace {

bcs_status read_int(Solver* s, const int32_t* d, int32_t* h) {
  BCS_CU(s, cudaMemcpyAsync(h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  return BCS_OK;
}

bcs_status max_of(Solver* s, const int32_t* a, int n, int32_t* out) {
  DBuf<int32_t> m;
  BCS_ALLOC(s, m, 1);
  BCS_CU(s, cudaMemsetAsync(m.p, 0, sizeof(int32_t), s->stream));
  if (n > 0) BCS_LAUNCH_DEP(s, K_SETUP_GAL, 0, 0, k_max_int, grid_for(n, 256) < 1024 ? grid_for(n, 256) : 1024, 256, 0, n, a, m.p);
  return read_int(s, m.p, out);
}

// h[0] = *d_total, h[1] = max of a[0..n) (n >= 0, values >= 0), one sync.
bcs_status total_and_max(Solver* s, const int32_t* d_total, const int32_t* a, int n, int32_t* h) {
  DBuf<int32_t> m;
  BCS_ALLOC(s, m, 2);
  BCS_CU(s, cudaMemsetAsync(m.p, 0, 2 * sizeof(int32_t), s->stream));
  if (n > 0)
    BCS_LAUNCH_DEP(s, K_SETUP_GAL, 0, 0, k_max_int, grid_for(n, 256) < 1024 ? grid_for(n, 256) : 1024, 256, 0, n, a,
               m.p + 1);
  BCS_CU(s, cudaMemcpyAsync(m.p, d_total, sizeof(int32_t), cudaMemcpyDeviceToDevice, s->stream));
  BCS_CU(s, cudaMemcpyAsync(h, m.p, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  return BCS_OK;
}

// Sorted unique pattern from per-row candidate segments. cnt[rows] holds the
// candidate counts on entry; fills out.rp / ci / nnz and crow (row of each
// nonzero).
template <class FillFn>
bcs_status pattern_from_candidates(Solver* s, int rows, DBuf<int32_t>& cnt, FillFn fill, Bsr& out,
                                   DBuf<int32_t>& crow) {
  DBuf<int32_t> cptr, cand;
  BCS_ALLOC(s, cptr, rows + 1);
  BCS_OKR(exclusive_scan(s, cnt.p, cptr.p, rows));
  int32_t tm[2] = {0, 0};
  BCS_OKR(total_and_max(s, cptr.p + rows, cnt.p, rows, tm));
  const int32_t total = tm[0], mx = tm[1];
  BCS_ALLOC(s, cand, total > 0 ? total : 1);
  BCS_OKR(fill(cptr.p, cand.p));
  BCS_OKR(segmented_sort_unique(s, cptr.p, cand.p, cnt.p, rows, mx));
  BCS_ALLOC(s, out.rp, rows + 1);
  BCS_OKR(exclusive_scan(s, cnt.p, out.rp.p, rows));
  BCS_OKR(total_and_max(s, out.rp.p + rows, cnt.p, rows, tm));
  const int32_t nnz = tm[0];
  out.rows = rows;
  out.nnz = nnz;
  out.maxrow = tm[1];
  BCS_ALLOC(s, out.ci, nnz > 0 ? nnz : 1);
  BCS_LAUNCH_DEP(s, K_SETUP_GAL, 0, 0, k_compact, grid_for(rows, 256), 256, 0, rows, cptr.p, cand.p, out.rp.p,
             out.ci.p);
  BCS_ALLOC(s, crow, nnz > 0 ? nnz : 1);
  BCS_LAUNCH_DEP(s, K_SETUP_GAL, 0, 0, k_row_index, grid_for(rows, 256), 256, 0, rows, out.rp.p, crow.p);
  return BCS_OK;
}

// One matching pass on A (rows x rows): agg[rows]; returns the count.
// norms: A's block Frobenius norms when already known, else computed here.
// Also returns the aggregates' member counts (cnt[0..nagg), an array of
// rows entries) and their maximum, read back together with the count.
bcs_status match_pass(Solver* s, const Bsr& A, DBuf<int32_t>& agg, int* nagg, DBuf<int32_t>& cnt, int* maxmem,
                      const double* norms = nullptr) {
  const int rows = A.rows, nnz = A.nnz;
  DBuf<double> nrm, w;
  DBuf<int32_t> ridx, dpos, mate, choice, root, amin, flag, id;
  if (!norms) BCS_ALLOC(s, nrm, nnz);
  BCS_ALLOC(s, w, nnz);
  BCS_ALLOC(s, ridx, nnz);
  BCS_ALLOC(s, dpos, rows);
  BCS_ALLOC(s, mate, rows);
  BCS_ALLOC(s, choice, rows);
  BCS_ALLOC(s, root, rows);
  BCS_ALLOC(s, amin, rows);
  BCS_ALLOC(s, flag, rows);
  BCS_ALLOC(s, id, rows + 1);
  BCS_ALLOC(s, agg, rows);
  const unsigned gr = grid_for(rows, 256), gn = grid_for(nnz, 256);
  if (!norms) {
    BCS_OKR(with_n(s->n, [&](auto NC) -> bcs_status {
      constexpr int N = decltype(NC)::value;
      BCS_LAUNCH_DEP(s, K_SETUP_AGG, 8.0 * nnz * (N * N + 1), 2.0 * nnz * N * N, k_block_norms<N * N>, gn, 256, 0, nnz,
                 A.v.p, nrm.p);
      return BCS_OK;
    }));
  }
  BCS_LAUNCH_DEP(s, K_SETUP_AGG, 0, 0, k_row_index, gr, 256, 0, rows, A.rp.p, ridx.p);
  BCS_LAUNCH_DEP(s, K_SETUP_AGG, 0, 0, k_diag_pos, gr, 256, 0, rows, A.rp.p, A.ci.p, dpos.p, s->flag.p);
  BCS_LAUNCH_DEP(s, K_SETUP_AGG, 0, 0, k_weights, gn, 256, 0, nnz, A.rp.p, A.ci.p, ridx.p, dpos.p,
             norms ? norms : nrm.p, w.p);
  BCS_LAUNCH_DEP(s, K_SETUP_AGG, 0, 0, k_fill_int, gr, 256, 0, mate.p, rows, -1);
  // A round that pairs nobody leaves the state unchanged, so running every
  // round equals stopping at the first idle one.
  for (int round = 0; round < s->setup_cfg.matching_rounds; ++round) {
    BCS_LAUNCH_DEP(s, K_SETUP_AGG, 0, 0, k_choose, gr, 256, 0, rows, A.rp.p, A.ci.p, w.p, mate.p, choice.p);
    BCS_LAUNCH_DEP(s, K_SETUP_AGG, 0, 0, k_pair, gr, 256, 0, rows, choice.p, mate.p);
  }
  BCS_LAUNCH_DEP(s, K_SETUP_AGG, 0, 0, k_fill_int, gr, 256, 0, amin.p, rows, INT_MAX);
  BCS_LAUNCH_DEP(s, K_SETUP_AGG, 0, 0, k_root, gr, 256, 0, rows, A.rp.p, A.ci.p, w.p, mate.p, root.p, amin.p);
  BCS_LAUNCH_DEP(s, K_SETUP_AGG, 0, 0, k_is_min, gr, 256, 0, rows, root.p, amin.p, flag.p);
  BCS_OKR(exclusive_scan(s, flag.p, id.p, rows));
  BCS_LAUNCH_DEP(s, K_SETUP_AGG, 0, 0, k_assign, gr, 256, 0, rows, root.p, amin.p, id.p, agg.p);
  // member counts (aggregate ids are < rows) and their maximum, read with
  // the aggregate count in one round trip
  BCS_ALLOC(s, cnt, rows);
  DBuf<int32_t> hv;
  BCS_ALLOC(s, hv, 2);
  BCS_CU(s, cudaMemsetAsync(cnt.p, 0, (size_t)rows * sizeof(int32_t), s->stream));
  BCS_CU(s, cudaMemsetAsync(hv.p, 0, 2 * sizeof(int32_t), s->stream));
  BCS_LAUNCH_DEP(s, K_SETUP_AGG, 0, 0, k_count_by, gr, 256, 0, rows, agg.p, cnt.p);
  BCS_LAUNCH_DEP(s, K_SETUP_AGG, 0, 0, k_max_int, gr < 1024 ? gr : 1024, 256, 0, rows, cnt.p, hv.p + 1);
  BCS_CU(s, cudaMemcpyAsync(hv.p, id.p + rows, sizeof(int32_t), cudaMemcpyDeviceToDevice, s->stream));
  int32_t h[2] = {0, 0};
  BCS_CU(s, cudaMemcpyAsync(h, hv.p, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  *nagg = h[0];
  *maxmem = h[1];
  return BCS_OK;
}

// Member lists of an aggregation: mptr[nagg+1], mem (members ascending).
// cnt[0..nagg): member counts from match_pass (overwritten), mx their maximum.
bcs_status members(Solver* s, int rows, int nagg, const int32_t* agg, int32_t* cnt, int mx, DBuf<int32_t>& mptr,
                   DBuf<int32_t>& mem) {
  DBuf<int32_t> cursor;
  BCS_ALLOC(s, cursor, nagg);
  BCS_ALLOC(s, mptr, nagg + 1);
  BCS_ALLOC(s, mem, rows);
  BCS_CU(s, cudaMemsetAsync(cursor.p, 0, nagg * sizeof(int32_t), s->stream));
  if (mx > 4096) BCS_OKR(max_of(s, cnt, nagg, &mx));  // a loose bound: the sort wants the real length
  BCS_OKR(exclusive_scan(s, cnt, mptr.p, nagg));
  BCS_LAUNCH_DEP(s, K_SETUP_GAL, 0, 0, k_place_by, grid_for(rows, 256), 256, 0, rows, agg, (const int32_t*)nullptr,
             mptr.p, cursor.p, mem.p);
  // members are distinct: sort/unique keeps the counts and sorts each list
  return segmented_sort_unique(s, mptr.p, mem.p, cnt, nagg, mx);
}

// Pattern of A_c = P_tent^T A P_tent (row I: sorted aggregates of its
// members' columns) and the plan of k_tent_sum (per coarse row its fine
// blocks in position order and each one's output block), from one segmented
// sort of packed (coarse column, sequence index) candidates. Sets A_c.maxrow.
// Two host reads.
// maxmem: the largest aggregate; with A.maxrow known, maxmem * A.maxrow
// bounds the longest candidate segment and its read is skipped.
bcs_status tent_pattern(Solver* s, const Bsr& A, int nagg, const int32_t* agg, const int32_t* mptr,
                        const int32_t* mem, int maxmem, Bsr& Ac, TentPlan& plan) {
  DBuf<int32_t> cnt, hv, moff;
  BCS_ALLOC(s, cnt, nagg);
  BCS_ALLOC(s, plan.seg, nagg + 1);
  BCS_ALLOC(s, hv, 4);
  BCS_ALLOC(s, moff, A.rows);
  BCS_CU(s, cudaMemsetAsync(hv.p, 0, 4 * sizeof(int32_t), s->stream));
  BCS_LAUNCH_DEP(s, K_SETUP_GAL, 0, 0, k_cand_count_tent, grid_for(nagg, 256), 256, 0, nagg, mptr, mem, A.rp.p, cnt.p,
             moff.p, hv.p + 1);
  BCS_OKR(exclusive_scan(s, cnt.p, plan.seg.p, nagg));
  int32_t h[2] = {0, 0};
  int max_c;
  if (A.maxrow >= 0 && maxmem > 0 && (long long)maxmem * A.maxrow <= 4096) {
    max_c = maxmem * A.maxrow;
  } else {
    BCS_CU(s, cudaMemcpyAsync(h, hv.p, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
    BCS_CU(s, cudaStreamSynchronize(s->stream));
    max_c = h[1];
  }
  DBuf<uint64_t> cand;
  BCS_ALLOC(s, cand, A.nnz);
  BCS_ALLOC(s, plan.sk, A.nnz);
  BCS_LAUNCH_DEP(s, K_SETUP_GAL, 16.0 * A.nnz, 0, k_cand_pack_tent, grid_for(A.rows, 256), 256, 0, A.rows, A.rp.p,
             A.ci.p, agg, plan.seg.p, moff.p, cand.p);
  BCS_OKR(segmented_sort64(s, plan.seg.p, cand.p, nagg, max_c));
  BCS_LAUNCH_DEP(s, K_SETUP_GAL, 12.0 * A.nnz, 0, k_runs_count, std::min<unsigned>(grid_for(nagg, 8), RC_BLOCKS), 256,
             0, nagg, plan.seg.p, cand.p,
             cnt.p, hv.p + 3);
  BCS_ALLOC(s, Ac.rp, nagg + 1);
  BCS_OKR(exclusive_scan(s, cnt.p, Ac.rp.p, nagg));
  BCS_CU(s, cudaMemcpyAsync(hv.p + 2, Ac.rp.p + nagg, sizeof(int32_t), cudaMemcpyDeviceToDevice, s->stream));
  BCS_CU(s, cudaMemcpyAsync(h, hv.p + 2, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  Ac.rows = Ac.cols = nagg;
  Ac.nnz = h[0];
  Ac.maxrow = h[1];
  BCS_ALLOC(s, Ac.ci, Ac.nnz);
  BCS_LAUNCH_DEP(s, K_SETUP_GAL, 12.0 * A.nnz + 4.0 * Ac.nnz, 0, k_runs_emit, grid_for((size_t)nagg * 32, 256), 256, 0,
             nagg, plan.seg.p, cand.p, Ac.rp.p, Ac.ci.p, plan.sk.p);
  return BCS_OK;
}

bcs_status tent_values(Solver* s, const Bsr& A, const TentPlan& plan, Bsr& Ac) {
  const int n = s->n;
  BCS_ALLOC(s, Ac.v, (size_t)Ac.nnz * n * n);
  return with_n(n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    using S = TentShape<N * N>;
    if ((size_t)Ac.nnz * N * N >= (1ull << 31)) return s->fail(BCS_EINVAL, "Galerkin product too large");
    const int nagg = Ac.rows;
    const unsigned grid = grid_for(nagg, TS_WARPS * S::G);
    BCS_LAUNCH_DEP(s, K_SETUP_GAL, 8.0 * (A.nnz + Ac.nnz) * N * N + 4.0 * A.nnz + 4.0 * (nagg + 1) * 2,
               1.0 * (A.nnz - Ac.nnz) * N * N, k_tent_sum<N * N>, grid, TS_WARPS * 32, 0, nagg, plan.seg.p,
               plan.sk.p, Ac.rp.p, A.v.p, Ac.v.p);
    return BCS_OK;
  });
}

// Aggregation with agg_passes matching passes; fills L.agg / L.nagg.
bcs_status aggregate_level(Solver* s, Level& L, const double* norms) {
  int nagg = 0, maxmem = 0;
  DBuf<int32_t> cnt;
  BCS_OKR(match_pass(s, L.A, L.agg, &nagg, cnt, &maxmem, norms));
  DBuf<int32_t> cur_agg;
  BCS_ALLOC(s, cur_agg, L.A.rows);
  BCS_CU(s, cudaMemcpyAsync(cur_agg.p, L.agg.p, L.A.rows * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                            s->stream));
  Bsr G;  // current aggregate graph (passes >= 2)
  const Bsr* cur = &L.A;
  for (int pass = 1; pass < s->setup_cfg.agg_passes; ++pass) {
    DBuf<int32_t> mptr, mem;
    BCS_OKR(members(s, cur->rows, nagg, cur_agg.p, cnt.p, maxmem, mptr, mem));
    Bsr Abar;
    TentPlan plan;
    BCS_OKR(tent_pattern(s, *cur, nagg, cur_agg.p, mptr.p, mem.p, maxmem, Abar, plan));
    BCS_OKR(tent_values(s, *cur, plan, Abar));
    DBuf<int32_t> a2;
    int n2 = 0, mm2 = 0;
    BCS_OKR(match_pass(s, Abar, a2, &n2, cnt, &mm2));
    // an aggregate of aggregates has at most the product of the largest
    // sizes (an upper bound is all the sorts need)
    maxmem = (int)std::min<long long>((long long)maxmem * mm2, L.A.rows);
    BCS_LAUNCH_DEP(s, K_SETUP_AGG, 0, 0, k_compose, grid_for(L.A.rows, 256), 256, 0, L.A.rows, a2.p, L.agg.p);
    cur_agg = std::move(a2);
    const bool stalled = n2 == nagg;
    nagg = n2;
    G = std::move(Abar);
    cur = &G;
    if (stalled) break;
  }
  L.nagg = nagg;
  // member counts of the final aggregates over the fine rows (recounted when
  // the graph was coarsened in between; maxmem is then an upper bound)
  if (cur != &L.A) {
    BCS_CU(s, cudaMemsetAsync(cnt.p, 0, (size_t)nagg * sizeof(int32_t), s->stream));
    BCS_LAUNCH_DEP(s, K_SETUP_AGG, 0, 0, k_count_by, grid_for(L.A.rows, 256), 256, 0, L.A.rows, L.agg.p, cnt.p);
  }
  L.cnt = std::move(cnt);
  L.maxmem = maxmem;
  return BCS_OK;
}

// Block inverses of level L: FP64 into L.dinv, or (fp32_inverses) FP32
// straight into L.dinv32. allocated: the output (and dpos) exist already.
bcs_status block_inverses(Solver* s, Level& L, bool full, bool allocated = false) {
  const int rows = L.A.rows, n = s->n;
  if (full || !L.dpos.p) {
    if (!allocated) BCS_ALLOC(s, L.dpos, rows);
    BCS_LAUNCH_DEP(s, K_SETUP_INV, 0, 0, k_diag_pos, grid_for(rows, 256), 256, 0, rows, L.A.rp.p, L.A.ci.p,
               L.dpos.p, s->flag.p);
  }
  const bool f32 = fp32_inverses(s);
  L.dinv64 = !f32;
  if (!allocated) {
    if (f32) BCS_ALLOC(s, L.dinv32, (size_t)rows * n * n);
    else BCS_ALLOC(s, L.dinv, (size_t)rows * n * n);
  }
  return with_n(n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    if (f32)
      BCS_LAUNCH_DEP(s, K_SETUP_INV, 12.0 * rows * N * N, 4.0 * rows * N * N * N, k_block_inverse32<N>,
                     grid_for(rows, 64), 64, 0, rows, L.dpos.p, L.A.v.p, L.dinv32.p, s->flag.p);
    else
      BCS_LAUNCH_DEP(s, K_SETUP_INV, 16.0 * rows * N * N, 4.0 * rows * N * N * N, k_block_inverse<N>,
                     grid_for(rows, 64), 64, 0, rows, L.dpos.p, L.A.v.p, L.dinv.p, s->flag.p);
    return BCS_OK;
  });
}

// Dense coarse inverses of at most this many unknowns run on one block in
// shared memory (16 N^2 bytes: 147 KB at 96).
constexpr int GJ_SMEM_MAX_N = 96;

bcs_status coarse_inverse(Solver* s, Level& L) {
  const int N = L.A.rows * s->n;
  s->cN = N;
  DBuf<double> M, colbuf;
  DBuf<int32_t> prow;
  BCS_ALLOC(s, M, (size_t)N * 2 * N);
  BCS_ALLOC(s, colbuf, 2 * (size_t)N);
  BCS_ALLOC(s, prow, N);
  BCS_ALLOC(s, s->cinv, (size_t)N * N);
  BCS_LAUNCH_DEP(s, K_SETUP_INV, 0, 0, k_dense_from_bsr, grid_for(L.A.rows, 64), 64, 0, L.A.rows, s->n, L.A.rp.p,
             L.A.ci.p, L.A.v.p, M.p, N);
  if (N <= GJ_SMEM_MAX_N) {
    // [A | I] fits one block's shared memory: no grid-wide barriers, no L2
    // round trip per pivot step
    const size_t smem = 16 * (size_t)N * N + N;
    BCS_CU(s, allow_max_dynamic_smem<k_gauss_jordan_smem>());
    BCS_LAUNCH_DEP(s, K_SETUP_INV, 24.0 * N * N * N, 3.0 * N * N * N, k_gauss_jordan_smem, 1, GJ_SMEM_THREADS, smem, N,
               M.p, prow.p, s->flag.p);
  } else {
    int dev = 0, sms = 0, per_sm = 0;
    BCS_CU(s, cudaGetDevice(&dev));
    BCS_CU(s, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256;
    const size_t smem = (size_t)N;
    BCS_CU(s, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gauss_jordan, threads, smem));
    if (per_sm < 1) return s->fail(BCS_ECUDA, "coarse inverse kernel cannot be resident");
    int blocks = sms * per_sm;
    if (blocks > N) blocks = N;
    int Nn = N;
    double* Mp = M.p;
    double* cb = colbuf.p;
    int32_t* pr = prow.p;
    int32_t* fl = s->flag.p;
    void* args[] = {&Nn, &Mp, &cb, &pr, &fl};
    s->pre(K_SETUP_INV);
    BCS_CU(s, cudaLaunchCooperativeKernel((void*)k_gauss_jordan, blocks, threads, args, smem, s->stream));
    BCS_OKR(s->post(K_SETUP_INV, "k_gauss_jordan", 24.0 * N * N * N, 3.0 * N * N * N));
  }
  BCS_LAUNCH_DEP(s, K_SETUP_INV, 0, 0, k_gj_finish, grid_for((size_t)N * N, 256), 256, 0, N, M.p, prow.p,
             s->cinv.p);
  return BCS_OK;
}

// R = P^T: structure (full) and values.
bcs_status transpose_P(Solver* s, Level& L, bool full) {
  Bsr& P = L.P;
  Bsr& R = L.R;
  const int rows = L.A.rows;
  if (full) {
    DBuf<int32_t> rcnt, cursor;
    R.rows = L.nagg;
    R.cols = rows;
    R.nnz = P.nnz;
    BCS_ALLOC(s, rcnt, L.nagg);
    BCS_ALLOC(s, cursor, L.nagg);
    BCS_ALLOC(s, R.rp, L.nagg + 1);
    BCS_ALLOC(s, R.ci, R.nnz);
    BCS_CU(s, cudaMemsetAsync(rcnt.p, 0, L.nagg * sizeof(int32_t), s->stream));
    BCS_CU(s, cudaMemsetAsync(cursor.p, 0, L.nagg * sizeof(int32_t), s->stream));
    BCS_LAUNCH_DEP(s, K_SETUP_GAL, 0, 0, k_count_by, grid_for(P.nnz, 256), 256, 0, P.nnz, P.ci.p, rcnt.p);
    BCS_OKR(exclusive_scan(s, rcnt.p, R.rp.p, L.nagg));
    BCS_LAUNCH_DEP(s, K_SETUP_GAL, 0, 0, k_place_by, grid_for(P.nnz, 256), 256, 0, P.nnz, P.ci.p, L.Prow.p, R.rp.p,
               cursor.p, R.ci.p);
    int32_t mx = 0;
    BCS_OKR(max_of(s, rcnt.p, L.nagg, &mx));
    BCS_OKR(segmented_sort_unique(s, R.rp.p, R.ci.p, rcnt.p, L.nagg, mx));
    BCS_ALLOC(s, L.Rrow, R.nnz);
    BCS_LAUNCH_DEP(s, K_SETUP_GAL, 0, 0, k_row_index, grid_for(L.nagg, 256), 256, 0, L.nagg, R.rp.p, L.Rrow.p);
  }
  const int n = s->n;
  BCS_ALLOC(s, R.v, (size_t)R.nnz * n * n);
  return with_n(n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    BCS_LAUNCH_DEP(s, K_SETUP_GAL, 16.0 * R.nnz * N * N, 0, k_transpose_values<N>, grid_for(R.nnz, 128), 128, 0,
               R.nnz, L.Rrow.p, R.ci.p, P.rp.p, P.ci.p, P.v.p, R.v.p);
    return BCS_OK;
  });
}

// Smoothed prolongation of level L: omega_P, pattern (full), values, R.
bcs_status smoothed_prolongation(Solver* s, Level& L, bool full) {
  const int rows = L.A.rows, n = s->n;
  DBuf<double> rho;
  BCS_ALLOC(s, rho, 1);
  BCS_CU(s, cudaMemsetAsync(rho.p, 0, sizeof(double), s->stream));
  BCS_OKR(with_n(n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    BCS_LAUNCH_DEP(s, K_SETUP_GAL, 8.0 * L.A.nnz * N * N, 2.0 * L.A.nnz * N * N * N, k_rho<N>, grid_for(rows, 128),
               128, 0, rows, L.A.rp.p, L.A.v.p, L.dinv.p, rho.p);
    return BCS_OK;
  }));
  double h_rho = 0.0;
  BCS_CU(s, cudaMemcpyAsync(&h_rho, rho.p, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  L.omega_p = s->setup_cfg.p_omega / h_rho;
  if (full) {
    DBuf<int32_t> cnt;
    BCS_ALLOC(s, cnt, rows);
    BCS_LAUNCH_DEP(s, K_SETUP_GAL, 0, 0, k_cand_count_p, grid_for(rows, 256), 256, 0, rows, L.A.rp.p, cnt.p);
    auto fill = [&](const int32_t*, int32_t* cand) -> bcs_status {
      // candidate segments coincide with A's rows
      BCS_LAUNCH_DEP(s, K_SETUP_GAL, 0, 0, k_cand_fill_p, grid_for(rows, 256), 256, 0, rows, L.A.rp.p, L.A.ci.p,
                 L.agg.p, cand);
      return BCS_OK;
    };
    BCS_OKR(pattern_from_candidates(s, rows, cnt, fill, L.P, L.Prow));
    L.P.cols = L.nagg;
  }
  BCS_ALLOC(s, L.P.v, (size_t)L.P.nnz * n * n);
  const double om = L.omega_p;
  BCS_OKR(with_n(n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    BCS_LAUNCH_DEP(s, K_SETUP_GAL, 8.0 * (L.A.nnz + L.P.nnz) * N * N, 2.0 * L.P.nnz * N * N * N, k_p_values<N>,
               grid_for(L.P.nnz, 128), 128, 0, L.P.nnz, L.Prow.p, L.P.ci.p, L.A.rp.p, L.A.ci.p, L.A.v.p, L.dinv.p,
               L.agg.p, om, L.P.v.p);
    return BCS_OK;
  }));
  return transpose_P(s, L, full);
}

// C = A B (block SpGEMM): pattern when full, values always.
bcs_status spgemm(Solver* s, const Bsr& A, const Bsr& B, Bsr& Cm, DBuf<int32_t>& crow, bool full) {
  const int rows = A.rows, n = s->n;
  if (full) {
    DBuf<int32_t> cnt;
    BCS_ALLOC(s, cnt, rows);
    BCS_LAUNCH_DEP(s, K_SETUP_GAL, 0, 0, k_cand_count_gemm, grid_for(rows, 256), 256, 0, rows, A.rp.p, A.ci.p, B.rp.p,
               cnt.p);
    auto fill = [&](const int32_t* cptr, int32_t* cand) -> bcs_status {
      BCS_LAUNCH_DEP(s, K_SETUP_GAL, 0, 0, k_cand_fill_gemm, grid_for(rows, 256), 256, 0, rows, A.rp.p, A.ci.p,
                 B.rp.p, B.ci.p, cptr, cand);
      return BCS_OK;
    };
    BCS_OKR(pattern_from_candidates(s, rows, cnt, fill, Cm, crow));
    Cm.cols = B.cols;
  }
  BCS_ALLOC(s, Cm.v, (size_t)Cm.nnz * n * n);
  return with_n(n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    BCS_LAUNCH_DEP(s, K_SETUP_GAL, 8.0 * (A.nnz + Cm.nnz) * N * N, 0, k_gemm_values<N>, grid_for(Cm.nnz, 64), 64, 0,
               Cm.nnz, crow.p, Cm.ci.p, A.rp.p, A.ci.p, A.v.p, B.rp.p, B.ci.p, B.v.p, Cm.v.p);
    return BCS_OK;
  });
}

bcs_status check_flags(Solver* s, bool* singular) {
  int32_t h = 0;
  BCS_OKR(read_int(s, s->flag.p, &h));
  *singular = false;
  if (h & 4) return s->fail(BCS_EINVAL, "a block row has no diagonal block");
  if (h & (8 | 16)) *singular = true;
  return BCS_OK;
}

// Transfer operators and coarse matrix for level l -> l+1.
bcs_status build_transfer(Solver* s, int l, bool full) {
  if ((int)s->lv.size() <= l + 1) s->lv.emplace_back();
  Level& L = s->lv[l];
  Level& Lc = s->lv[l + 1];
  if (full) {
    BCS_OKR(members(s, L.A.rows, L.nagg, L.agg.p, L.cnt.p, L.maxmem, L.mptr, L.mem));
    L.cnt.release();
  }
  if (s->setup_cfg.pmode == BCS_P_TENTATIVE) {
    if (full) BCS_OKR(tent_pattern(s, L.A, L.nagg, L.agg.p, L.mptr.p, L.mem.p, L.maxmem, Lc.A, L.tent));
    BCS_OKR(tent_values(s, L.A, L.tent, Lc.A));
  } else {
    BCS_OKR(smoothed_prolongation(s, L, full));
    BCS_OKR(spgemm(s, L.A, L.P, L.AP, L.AProw, full));
    BCS_OKR(spgemm(s, L.R, L.AP, Lc.A, L.Crow, full));
  }
  Lc.A.cols = Lc.A.rows;
  return BCS_OK;
}

}  // namespace

bcs_status amg_setup_levels(Solver* s, bool full);

bool fp32_inverses(const Solver* s) {
  const bcs_config& c = s->setup_cfg;
  // FP64 inverses are read by the FP64 cycle, the block-Jacobi
  // preconditioner (applied in FP64) and smoothed P's damping estimate
  return c.precision != BCS_PREC_FP64 && c.precond != BCS_PC_JACOBI &&
         !(c.precond == BCS_PC_AMG && c.pmode == BCS_P_SMOOTHED);
}

bcs_status level_dinv64(Solver* s, int l, const double** out, DBuf<double>& tmp) {
  Level& L = s->lv[l];
  if (L.dinv64) {
    *out = L.dinv.p;
    return BCS_OK;
  }
  const int rows = L.A.rows, n = s->n;
  BCS_ALLOC(s, tmp, (size_t)rows * n * n);
  BCS_OKR(with_n(n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    BCS_LAUNCH_DEP(s, K_SETUP_INV, 16.0 * rows * N * N, 4.0 * rows * N * N * N, k_block_inverse<N>,
                   grid_for(rows, 64), 64, 0, rows, L.dpos.p, L.A.v.p, tmp.p, s->flag.p);
    return BCS_OK;
  }));
  *out = tmp.p;
  return BCS_OK;
}

bcs_status amg_setup(Solver* s, bool full) {
  const bcs_status st = amg_setup_levels(s, full);
  s->nrm0_fresh = false;  // the norms belong to these values only
  return st;
}

bcs_status amg_setup_levels(Solver* s, bool full) {
  const bcs_config& cfg = s->setup_cfg;
  if (full) {
    s->lv.resize(1);
    Level& L0 = s->lv[0];
    L0.agg.release();
    L0.nagg = 0;
    L0.coarse_kind = -1;
  }
  BCS_CU(s, cudaMemsetAsync(s->flag.p, 0, 4 * sizeof(int32_t), s->stream));
  // With block Jacobi, a singular diagonal block leaves only garbage values
  // behind (no index depends on them), so the flags are read once, at the
  // end; the multicolour factorisations read them per level.
  const bool dilu = cfg.precond == BCS_PC_SGS || (cfg.precond == BCS_PC_AMG && cfg.smoother != BCS_SMOOTH_JACOBI);
  // With block Jacobi a level's block inverses (FP64-bound) do not depend on
  // its aggregation (latency-bound small kernels) or, at a values-only
  // resetup, on its Galerkin product: they run on a second stream beside
  // them and are joined before anything reads them (the FP32 copies,
  // smoothed prolongation, the flags at the end).
  const bool side = !dilu && cfg.pmode == BCS_P_TENTATIVE;
  if (side && !s->sstream) BCS_CU(s, cudaStreamCreateWithFlags(&s->sstream, cudaStreamNonBlocking));
  if (side && !s->sev[0]) {
    BCS_CU(s, cudaEventCreateWithFlags(&s->sev[0], cudaEventDisableTiming));
    BCS_CU(s, cudaEventCreateWithFlags(&s->sev[1], cudaEventDisableTiming));
  }
  bool forked = false;
  for (int l = 0;; ++l) {
    Level& L = s->lv[l];
    LevelScope level_scope(s, l);
    if (side) {
      // buffers first, stream-ordered on the solver's stream
      BCS_ALLOC(s, L.dpos, L.A.rows);
      if (fp32_inverses(s)) BCS_ALLOC(s, L.dinv32, (size_t)L.A.rows * s->n * s->n);
      else BCS_ALLOC(s, L.dinv, (size_t)L.A.rows * s->n * s->n);
      BCS_CU(s, cudaEventRecord(s->sev[0], s->stream));
      BCS_CU(s, cudaStreamWaitEvent(s->sstream, s->sev[0], 0));
      const cudaStream_t own = s->stream;
      s->stream = s->sstream;
      const bcs_status st_inv = block_inverses(s, L, full, true);
      s->stream = own;
      BCS_OKR(st_inv);
      forked = true;
    } else {
      BCS_OKR(block_inverses(s, L, full));
    }
    if (dilu) {
      bool singular = false;
      BCS_OKR(check_flags(s, &singular));
      if (singular) return s->fail(BCS_SINGULAR_BLOCK, "singular diagonal block at level " + std::to_string(l));
      BCS_OKR(dilu_setup(s, L, full, cfg.precond == BCS_PC_SGS || cfg.smoother == BCS_SMOOTH_SGS));
    }
    bool last;
    if (full) {
      const int C = L.A.rows;
      last = C <= cfg.coarse_size || l == cfg.max_levels - 1 || cfg.precond != BCS_PC_AMG;
      if (!last) {
        BCS_OKR(aggregate_level(s, L, l == 0 && s->nrm0_fresh ? s->nrm0.p : nullptr));
        if (L.nagg >= C || (double)L.nagg > cfg.max_coarsen_ratio * C) {
          last = true;
          L.agg.release();
          L.nagg = 0;
        }
      }
    } else {
      last = L.coarse_kind >= 0;
    }
    if (last) {
      s->lv.resize(l + 1);
      Level& Lf = s->lv[l];
      if (cfg.precond != BCS_PC_AMG) {
        Lf.coarse_kind = 1;
      } else if ((long long)Lf.A.rows * s->n <= cfg.coarse_dense_max) {
        Lf.coarse_kind = 0;
        BCS_OKR(coarse_inverse(s, Lf));
      } else {
        Lf.coarse_kind = 1;
        s->cinv.release();
        s->cN = 0;
      }
      break;
    }
    L.coarse_kind = -1;
    BCS_OKR(build_transfer(s, l, full));
  }
  if (forked) {  // join the second stream
    BCS_CU(s, cudaEventRecord(s->sev[1], s->sstream));
    BCS_CU(s, cudaStreamWaitEvent(s->stream, s->sev[1], 0));
  }
  int32_t h = 0;
  BCS_OKR(read_int(s, s->flag.p, &h));
  if (h & 4) return s->fail(BCS_EINVAL, "a block row has no diagonal block");
  if (h & 8) return s->fail(BCS_SINGULAR_BLOCK, "singular diagonal block");
  if (h & 16) return s->fail(BCS_SINGULAR_BLOCK, "singular coarsest-level matrix");
  return BCS_OK;
}

}  // namespace bcs
