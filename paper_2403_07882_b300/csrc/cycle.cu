// Block-CSR row kernels (SpMV, residual, damped block-Jacobi sweep), the
// outer FP64 SpMV (Eq. 1's left-hand side y_i = sum_j A_ij x_j), the
// inter-grid transfers and the AMG V-cycle built from them.
//
// Row mapping: a warp serves floor(32 / n) block rows; lane l handles scalar
// row r = l % n of block row l / n. The n lanes of a block row sit in one warp
// and exchange residual components by shuffle for the D^-1 epilogue. Each lane
// reads its row of every block (n contiguous values) and the matching x
// block, one fma per matrix entry.
//
// V-cycle (reading of the paper's unparameterised "AMG preconditioner"):
// per level, nu1 damped block-Jacobi sweeps x <- x + w D^-1 (b - A x) (the
// first from x = 0 is x = w D^-1 b), residual, restriction R = P^T,
// recursion, prolongation-correction, nu2 sweeps; the coarsest level applies
// its dense FP64 inverse (or smoother sweeps when too large for one).
#include <cooperative_groups.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>

#include "internal.h"

namespace bcs {

namespace {

template <class AT, class T> __device__ __forceinline__ AT lda(const T* p);
template <> __device__ __forceinline__ double lda<double, double>(const double* p) { return __ldg(p); }
template <> __device__ __forceinline__ double lda<double, float>(const float* p) { return (double)__ldg(p); }
template <> __device__ __forceinline__ float lda<float, float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float lda<float, bf16>(const bf16* p) { return __bfloat162float(__ldg(p)); }

template <int N>
struct RowMap {
  static constexpr int RPW = 32 / N;  // block rows per warp
  int rw, r, i;
  bool active;
  __device__ explicit RowMap(int rows) {
    const int lane = threadIdx.x & 31;
    rw = lane / N;
    r = lane - rw * N;
    const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    i = warp * RPW + rw;
    active = rw < RPW && i < rows;
  }
};

template <int N, class AT, class TV, class TX>
__device__ __forceinline__ AT row_dot(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                      const TV* __restrict__ val, const TX* __restrict__ x, int i, int r) {
  AT acc = 0;
  const int kb = __ldg(rp + i), ke = __ldg(rp + i + 1);
#pragma unroll 2
  for (int k = kb; k < ke; ++k) {
    const int j = __ldg(ci + k);
    const TV* a = val + (size_t)k * (N * N) + r * N;
    const TX* xj = x + (size_t)j * N;
#pragma unroll
    for (int c = 0; c < N; ++c) acc = fma(lda<AT>(a + c), lda<AT>(xj + c), acc);
  }
  return acc;
}

// y = A x (M_SPMV), y += A x (M_ADD), y = b - A x (M_RESID).
template <int N, class AT, class TV, class TX, class TY, int MODE>
__device__ __forceinline__ void rows_eval(int i, int r, const int32_t* __restrict__ rp,
                                          const int32_t* __restrict__ ci, const TV* __restrict__ val,
                                          const TX* __restrict__ x, TY* __restrict__ y, const TY* __restrict__ b) {
  const AT acc = row_dot<N, AT>(rp, ci, val, x, i, r);
  const size_t o = (size_t)i * N + r;
  if (MODE == M_SPMV) y[o] = (TY)acc;
  else if (MODE == M_ADD) y[o] = (TY)((AT)y[o] + acc);
  else y[o] = (TY)((AT)b[o] - acc);
}

template <int N, class AT, class TV, class TX, class TY, int MODE>
__global__ void __launch_bounds__(128) k_rows(int rows, const int32_t* __restrict__ rp,
                                              const int32_t* __restrict__ ci, const TV* __restrict__ val,
                                              const TX* __restrict__ x, TY* __restrict__ y,
                                              const TY* __restrict__ b) {
  dep_enter();
  RowMap<N> m(rows);
  if (!m.active) return;
  rows_eval<N, AT, TV, TX, TY, MODE>(m.i, m.r, rp, ci, val, x, y, b);
}

// ---- multicolour DILU sweeps (one launch per colour) -------------------------
// Rows of colour c (slots t0 .. t0 + cnt of the colour lists crow), lane
// (w, r) = scalar row r of the w-th row.
// Forward:  y_i = E_i^{-1} (r_i - sum_{colour(j) < c} A_ij y_j).
// Backward: d_i = y_i - E_i^{-1} sum_{colour(j) > c} A_ij d_j;  x_i += d_i.
// The blocks come from the row's split lists (lower part forward, upper part
// backward, each in column order: the same fma sequence as a walk over the
// whole row that skips the other blocks, without reading their colours).
// GATHER: val is the BSR array, indexed through dsrc (FP64 cycle); else val
// holds the split blocks in split order. One row of a colour's sweep: lane
// (rw, r) of a row group; every lane of the warp calls it (shuffles), active
// says whether the lane has a row. Vectors the sweeps write (r, y, d, x) are
// read with ordinary loads.
// COH: the vectors are read through L2 (ld.global.cg), for the one-launch
// step in which other blocks of the cluster wrote them in earlier phases.
template <bool COH, class T>
__device__ __forceinline__ T ldw(const T* p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}

template <int N, class AT, class TV, class TD, class TC, bool FWD, bool GATHER, bool COH = false>
__device__ __forceinline__ void dilu_row(bool active, int i, int t, int rw, int r, const int32_t* __restrict__ dptr,
                                         const int32_t* __restrict__ dmid, const int32_t* __restrict__ dsrc,
                                         const int32_t* __restrict__ dci, const TV* __restrict__ val,
                                         const TD* __restrict__ einv, const TC* rv, TC* y, TC* d, TC* x) {
  AT acc = 0;
  if (active) {
    const int qb = FWD ? __ldg(dptr + t) : __ldg(dmid + t);
    const int qe = FWD ? __ldg(dmid + t) : __ldg(dptr + t + 1);
    for (int q = qb; q < qe; ++q) {
      const int j = __ldg(dci + q);
      const size_t blk = GATHER ? (size_t)__ldg(dsrc + q) : (size_t)q;
      const TV* a = val + blk * (N * N) + r * N;
      const TC* v = (FWD ? y : d) + (size_t)j * N;
#pragma unroll
      for (int cc = 0; cc < N; ++cc) acc = fma(lda<AT>(a + cc), (AT)ldw<COH>(v + cc), acc);
    }
  }
  const size_t o = (size_t)i * N + r;
  const AT u = active ? (FWD ? (AT)ldw<COH>(rv + o) - acc : acc) : (AT)0;
  AT s = 0;
#pragma unroll
  for (int cc = 0; cc < N; ++cc) {
    const AT tc = __shfl_sync(0xffffffffu, u, (rw * N + cc) & 31);
    if (active) s = fma(lda<AT>(einv + o * N + cc), tc, s);
  }
  if (!active) return;
  if (FWD) {
    y[o] = (TC)s;
  } else {
    const AT dv = (AT)ldw<COH>(y + o) - s;
    d[o] = (TC)dv;
    x[o] = (TC)((AT)ldw<COH>(x + o) + dv);
  }
}

template <int N, class AT, class TV, class TD, class TC, bool FWD, bool GATHER>
__global__ void __launch_bounds__(128) k_dilu_sweep(int cnt, int t0, const int32_t* __restrict__ crow,
                                                    const int32_t* __restrict__ dptr,
                                                    const int32_t* __restrict__ dmid,
                                                    const int32_t* __restrict__ dsrc,
                                                    const int32_t* __restrict__ dci, const TV* __restrict__ val,
                                                    const TD* __restrict__ einv, const TC* __restrict__ r,
                                                    TC* __restrict__ y, TC* __restrict__ d, TC* __restrict__ x) {
  dep_enter();
  RowMap<N> m(cnt);
  const int t = t0 + (m.active ? m.i : 0);
  const int i = m.active ? __ldg(crow + t) : 0;
  dilu_row<N, AT, TV, TD, TC, FWD, GATHER>(m.active, i, t, m.rw, m.r, dptr, dmid, dsrc, dci, val, einv, r, y, d,
                                           x);
}

// ---- sliced (SELL) copy for the FP32 / BF16 cycle ---------------------------
// A slice is floor(32/n) consecutive block rows served by one warp (lane l:
// scalar row r = l % n of block row rw = l / n). Step t of a slice holds the
// k-th block of each of its rows, stored column-major so that for a fixed
// column c the warp reads one contiguous run: value (rw, r, c) of step t sits
// at t * n*n*RPW + (c * RPW + rw) * n + r. Rows shorter than the slice's
// longest are padded (the padding is skipped). Each lane loads one component
// of its row's x block and the row's lanes exchange them by shuffle.
__global__ void k_slice_len(int rows, int rpw, int nslices, const int32_t* __restrict__ rp,
                            const int32_t* __restrict__ order, int32_t* __restrict__ slen) {
  dep_enter();
  const int sl = blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= nslices) return;
  int m = 0;
  for (int rw = 0; rw < rpw; ++rw) {
    const int pos = sl * rpw + rw;
    if (pos >= rows) break;
    const int i = order ? order[pos] : pos;
    m = max(m, rp[i + 1] - rp[i]);
  }
  slen[sl] = m;
}

// One warp per slice, the same lane mapping as the sweep: lane (w, r) reads
// row r of each block of row w (the n lanes of a row cover the block's
// contiguous span) and writes it column-major, so for a fixed column the
// warp writes one contiguous run.
template <int N, class TV>
__global__ void k_slice_fill(int rows, int nslices, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const double* __restrict__ val, const int32_t* __restrict__ sptr, int32_t* __restrict__ sci,
                             TV* __restrict__ sv) {
  dep_enter();
  constexpr int NN = N * N, RPW = 32 / N, TILE = NN * RPW;
  const int lane = threadIdx.x & 31;
  const int w = lane / N, r = lane - w * N;
  const int sl = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (sl >= nslices) return;
  const int i = sl * RPW + w;
  const bool active = w < RPW && i < rows;
  const int p0 = active ? rp[i] : 0, len = active ? rp[i + 1] - p0 : 0;
  const int t0 = sptr[sl];
  for (int k = 0; k < len; ++k) {
    const int p = p0 + k;
    const double* a = val + (size_t)p * NN + r * N;
    TV* tile = sv + (size_t)(t0 + k) * TILE;
#pragma unroll
    for (int c = 0; c < N; ++c) {
      if constexpr (std::is_same<TV, bf16>::value) tile[c * RPW * N + lane] = __double2bfloat16(a[c]);
      else tile[c * RPW * N + lane] = (TV)a[c];
    }
    if (r == 0) sci[(size_t)(t0 + k) * RPW + w] = ci[p];
  }
}

__device__ __forceinline__ float ldsv(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldsv(const bf16* p) { return __bfloat162float(__ldg(p)); }

constexpr int SELL_U = 4;  // steps per chunk of the lane-per-row kernels

// Vector loads: the read-only path for vectors that no other block of the
// same launch writes; the L2 path (coherent across the SMs of a cluster) in
// the coarse-tail kernel, where earlier phases of the same launch wrote them.
template <bool COH>
__device__ __forceinline__ float ldvec(const float* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}

template <int N, class TV, bool JACOBI, bool COH>
__device__ __forceinline__ void sell_slice(int sl, int rows, const int32_t* __restrict__ rp,
                                           const int32_t* __restrict__ sptr, const int32_t* __restrict__ sci,
                                           const TV* __restrict__ sv, const float* __restrict__ dinv,
                                           const float* x, const float* b, float* y, float omega) {
  constexpr int RPW = 32 / N, NN = N * N, TILE = NN * RPW;
  const int lane = threadIdx.x & 31;
  const int rw = lane / N, r = lane - rw * N;
  const int i = sl * RPW + rw;
  const bool active = rw < RPW && i < rows;
  const size_t o = (size_t)i * N + r;
  const float bo = active ? ldvec<COH>(b + o) : 0.f;
  float xo = 0.f, d[N];
  if (JACOBI) {
    xo = active ? (COH ? __ldcg(x + o) : x[o]) : 0.f;
#pragma unroll
    for (int c = 0; c < N; ++c) d[c] = active ? __ldg(dinv + o * N + c) : 0.f;
  }
  const int len = active ? __ldg(rp + i + 1) - __ldg(rp + i) : 0;
  const int t0 = __ldg(sptr + sl), nt = __ldg(sptr + sl + 1) - t0;
  float acc = 0.f;
  for (int k0 = 0; k0 < nt; k0 += SELL_U) {
    int j[SELL_U];
    float xv[SELL_U], a[SELL_U][N];
#pragma unroll
    for (int u = 0; u < SELL_U; ++u) {
      const bool live = active && k0 + u < len;
      j[u] = live ? __ldg(sci + (size_t)(t0 + k0 + u) * RPW + rw) : 0;
    }
#pragma unroll
    for (int u = 0; u < SELL_U; ++u) xv[u] = (active && k0 + u < len) ? ldvec<COH>(x + (size_t)j[u] * N + r) : 0.f;
#pragma unroll
    for (int u = 0; u < SELL_U; ++u) {
      const TV* tile = sv + (size_t)(t0 + k0 + u) * TILE;
#pragma unroll
      for (int c = 0; c < N; ++c) a[u][c] = (active && k0 + u < len) ? ldsv(tile + c * RPW * N + lane) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < SELL_U; ++u)
#pragma unroll
      for (int c = 0; c < N; ++c) {
        const float xc = __shfl_sync(0xffffffffu, xv[u], (rw * N + c) & 31);
        if (active && k0 + u < len) acc = fmaf(a[u][c], xc, acc);
      }
  }
  if (!JACOBI) {
    if (active) y[o] = bo - acc;
    return;
  }
  const float res = active ? bo - acc : 0.f;
  float tt = 0.f;
#pragma unroll
  for (int c = 0; c < N; ++c) {
    const float rc = __shfl_sync(0xffffffffu, res, (rw * N + c) & 31);
    if (active) tt = fmaf(d[c], rc, tt);
  }
  if (active) y[o] = fmaf(omega, tt, xo);
}

// JACOBI: y = x + omega D^-1 (b - A x); otherwise y = b - A x. Same fma order
// as k_jacobi / k_rows (blocks in row order, columns ascending). Steps are
// consumed in chunks of SELL_U: the chunk's column indices are loaded
// together, then the x components they select, then the values, so a warp
// keeps several HBM round trips in flight instead of one per step; the
// epilogue's operands are loaded before the row loop.
template <int N, class TV, bool JACOBI>
__global__ void __launch_bounds__(128) k_sell(int rows, int nslices, const int32_t* __restrict__ rp,
                                              const int32_t* __restrict__ sptr, const int32_t* __restrict__ sci,
                                              const TV* __restrict__ sv, const float* __restrict__ dinv,
                                              const float* __restrict__ x, const float* __restrict__ b,
                                              float* __restrict__ y, float omega) {
  dep_enter();
  const int sl = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (sl >= nslices) return;  // uniform across the warp
  sell_slice<N, TV, JACOBI, false>(sl, rows, rp, sptr, sci, sv, dinv, x, b, y, omega);
}

// ---- thread-per-block-row layout (smap = 1) ---------------------------------
// Slices of 32 block rows, one warp each, one thread per block row. Step t of
// a slice holds the t-th block of each of its rows in a tile of n*n*32
// values, in groups of G = 16 bytes / value size consecutive block entries:
// group g of row w at t * n*n*32 + g * G * 32 + w * G, so a thread loads G
// entries with one 16-byte load and the warp's load is 512 contiguous bytes;
// the n*n mod G remaining entries are element-major after the groups. Rows
// shorter than their slice's longest are padded (the padding is skipped).
// Slice position p holds block row srow[p]: rows are taken in windows of
// SORT_WIN consecutive rows, longest first (ties by row index), so the rows
// of a slice have similar lengths and little padding (coarse levels mix rows
// of 7 to 30 blocks).
// (TprTile, in internal.h, gives these offsets.)

// resident blocks of 128 threads per SM the sweep is compiled for (caps its
// registers at 64)
#define TPR_MINB 7

// the NN entries of row w in one step tile, widened to FP32
template <int NN>
__device__ __forceinline__ void load_tile_row(const float* __restrict__ tile, int w, float* a) {
  using T = TprTile<NN, float>;
#pragma unroll
  for (int g = 0; g < T::NG; ++g) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(tile + g * 4 * 32 + w * 4));
    a[4 * g] = v.x;
    a[4 * g + 1] = v.y;
    a[4 * g + 2] = v.z;
    a[4 * g + 3] = v.w;
  }
#pragma unroll
  for (int r = 0; r < T::R; ++r) a[T::NG * 4 + r] = __ldg(tile + T::NG * 4 * 32 + r * 32 + w);
}

template <int NN>
__device__ __forceinline__ void load_tile_row(const bf16* __restrict__ tile, int w, float* a) {
  using T = TprTile<NN, bf16>;
#pragma unroll
  for (int g = 0; g < T::NG; ++g) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(tile + g * 8 * 32 + w * 8));
    const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u[k]));
      a[8 * g + 2 * k] = f.x;
      a[8 * g + 2 * k + 1] = f.y;
    }
  }
#pragma unroll
  for (int r = 0; r < T::R; ++r) a[T::NG * 8 + r] = __bfloat162float(__ldg(tile + T::NG * 8 * 32 + r * 32 + w));
}

constexpr int SORT_WIN = 256;

__global__ void __launch_bounds__(SORT_WIN) k_window_order(int rows, const int32_t* __restrict__ rp,
                                                          int32_t* __restrict__ srow) {
  dep_enter();
  __shared__ int len[SORT_WIN];
  const int w0 = blockIdx.x * SORT_WIN, i = w0 + threadIdx.x;
  const int cnt = min(SORT_WIN, rows - w0);
  const int li = i < rows ? rp[i + 1] - rp[i] : -1;
  len[threadIdx.x] = li;
  __syncthreads();
  if ((int)threadIdx.x >= cnt) return;
  int rank = 0;
  for (int j = 0; j < cnt; ++j) {
    const int lj = len[j];
    rank += (lj > li) || (lj == li && j < (int)threadIdx.x);
  }
  srow[w0 + rank] = i;
}

template <int N, class TV>
__global__ void k_tpr_fill(int rows, int nslices, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ val, const int32_t* __restrict__ srow,
                           const int32_t* __restrict__ sptr, int32_t* __restrict__ sci, TV* __restrict__ sv,
                           int32_t* __restrict__ tpos) {
  dep_enter();
  constexpr int NN = N * N;
  using T = TprTile<NN, TV>;
  const int lane = threadIdx.x & 31;
  const int sl = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (sl >= nslices) return;
  const int pos = sl * 32 + lane;
  const int i = pos < rows ? srow[pos] : 0;
  const int p0 = pos < rows ? rp[i] : 0, len = pos < rows ? rp[i + 1] - p0 : 0;
  const int t0 = sptr[sl];
  for (int k = 0; k < len; ++k) {
    const double* a = val + (size_t)(p0 + k) * NN;
    TV* tile = sv + (size_t)(t0 + k) * T::TILE;
    // one 16-byte store per group: the warp writes 512 contiguous bytes
#pragma unroll
    for (int g = 0; g < T::NG; ++g) {
      alignas(16) TV v[T::G];
#pragma unroll
      for (int q = 0; q < T::G; ++q) {
        if constexpr (std::is_same<TV, bf16>::value) v[q] = __double2bfloat16(a[g * T::G + q]);
        else v[q] = (TV)a[g * T::G + q];
      }
      *reinterpret_cast<uint4*>(tile + g * T::G * 32 + lane * T::G) = *reinterpret_cast<const uint4*>(v);
    }
#pragma unroll
    for (int r = 0; r < T::R; ++r) {
      if constexpr (std::is_same<TV, bf16>::value) tile[T::NG * T::G * 32 + r * 32 + lane] = __double2bfloat16(a[T::NG * T::G + r]);
      else tile[T::NG * T::G * 32 + r * 32 + lane] = (TV)a[T::NG * T::G + r];
    }
    sci[(size_t)(t0 + k) * 32 + lane] = ci[p0 + k];
    if (tpos) tpos[p0 + k] = (t0 + k) * 32 + lane;  // the slot of block-CSR position p0 + k
  }
}

// JACOBI: y = x + omega D^-1 (b - A x); otherwise y = b - A x. Per scalar row
// the fma sequence is the one of k_sell (blocks in row order, columns
// ascending; the epilogue in column order), so both layouts give identical
// results.
template <int N, class TV, bool JACOBI>
__device__ __forceinline__ void tpr_slice(int sl, int rows, const int32_t* __restrict__ rp,
                                             const int32_t* __restrict__ srow, const int32_t* __restrict__ sptr,
                                             const int32_t* __restrict__ sci, const TV* __restrict__ sv,
                                             const float* __restrict__ dinv, const float* __restrict__ x,
                                             const float* __restrict__ b, float* __restrict__ y, float omega) {
  constexpr int NN = N * N, TILE = NN * 32;
  const int lane = threadIdx.x & 31;
  const int pos = sl * 32 + lane;
  if (pos >= rows) return;
  const int i = __ldg(srow + pos);
  static_assert(TprTile<NN, TV>::TILE == TILE, "tile size");
  const int len = __ldg(rp + i + 1) - __ldg(rp + i);
  const int t0 = __ldg(sptr + sl);
  const size_t o = (size_t)i * N;
  float acc[N];
#pragma unroll
  for (int r = 0; r < N; ++r) acc[r] = 0.f;
  // software pipeline: the next step's column index and values are loaded
  // while the current step's x block arrives and is used
  float a[NN];
  int j = 0;
  if (len > 0) {
    j = __ldg(sci + (size_t)t0 * 32 + lane);
    load_tile_row<NN>(sv + (size_t)t0 * TILE, lane, a);
  }
  for (int k = 0; k < len; ++k) {
    float xv[N];
#pragma unroll
    for (int c = 0; c < N; ++c) xv[c] = __ldg(x + (size_t)j * N + c);
    float an[NN];
    int jn = 0;
    if (k + 1 < len) {
      jn = __ldg(sci + (size_t)(t0 + k + 1) * 32 + lane);
      load_tile_row<NN>(sv + (size_t)(t0 + k + 1) * TILE, lane, an);
    }
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
      for (int c = 0; c < N; ++c) acc[r] = fmaf(a[r * N + c], xv[c], acc[r]);
#pragma unroll
    for (int e = 0; e < NN; ++e) a[e] = an[e];
    j = jn;
  }
  if (!JACOBI) {
#pragma unroll
    for (int r = 0; r < N; ++r) y[o + r] = __ldg(b + o + r) - acc[r];
    return;
  }
  float res[N];
#pragma unroll
  for (int r = 0; r < N; ++r) res[r] = __ldg(b + o + r) - acc[r];
#pragma unroll
  for (int r = 0; r < N; ++r) {
    const float xo = x[o + r];
    float tt = 0.f;
#pragma unroll
    for (int c = 0; c < N; ++c) tt = fmaf(__ldg(dinv + (o + r) * N + c), res[c], tt);
    y[o + r] = fmaf(omega, tt, xo);
  }
}

template <int N, class TV, bool JACOBI>
__global__ void __launch_bounds__(128, TPR_MINB) k_tpr(int rows, int nslices, const int32_t* __restrict__ rp,
                                             const int32_t* __restrict__ srow, const int32_t* __restrict__ sptr,
                                             const int32_t* __restrict__ sci, const TV* __restrict__ sv,
                                             const float* __restrict__ dinv, const float* __restrict__ x,
                                             const float* __restrict__ b, float* __restrict__ y, float omega) {
  dep_enter();
  const int sl = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (sl >= nslices) return;
  tpr_slice<N, TV, JACOBI>(sl, rows, rp, srow, sptr, sci, sv, dinv, x, b, y, omega);
}

// y = x + omega D^-1 (b - A x)
template <int N, class AT, class TV, class TD, class TC>
__global__ void __launch_bounds__(128) k_jacobi(int rows, const int32_t* __restrict__ rp,
                                                const int32_t* __restrict__ ci, const TV* __restrict__ val,
                                                const TD* __restrict__ dinv, const TC* __restrict__ x,
                                                const TC* __restrict__ b, TC* __restrict__ y, AT omega) {
  dep_enter();
  RowMap<N> m(rows);
  AT res = 0;
  if (m.active) res = (AT)b[(size_t)m.i * N + m.r] - row_dot<N, AT>(rp, ci, val, x, m.i, m.r);
  AT t = 0;
#pragma unroll
  for (int c = 0; c < N; ++c) {
    const AT rc = __shfl_sync(0xffffffffu, res, (m.rw * N + c) & 31);
    if (m.active) t = fma((AT)dinv[((size_t)m.i * N + m.r) * N + c], rc, t);
  }
  if (m.active) {
    const size_t o = (size_t)m.i * N + m.r;
    y[o] = (TC)((AT)x[o] + omega * t);
  }
}

// y = omega D^-1 b (first sweep from a zero guess), element t = (i, r)
template <int N, class AT, class TD, class TC, bool COH>
__device__ __forceinline__ void jacobi0_elem(size_t t, const TD* __restrict__ dinv, const TC* b, TC* y, AT omega) {
  const size_t i = t / N;
  const int r = (int)(t - i * N);
  AT acc = 0;
#pragma unroll
  for (int c = 0; c < N; ++c) {
    AT bc;
    if constexpr (COH) bc = (AT)__ldcg(b + i * N + c);
    else bc = (AT)b[i * N + c];
    acc = fma((AT)dinv[(i * N + r) * N + c], bc, acc);
  }
  y[t] = (TC)(omega * acc);
}

template <int N, class AT, class TD, class TC>
__global__ void k_jacobi0(int rows, const TD* __restrict__ dinv, const TC* __restrict__ b, TC* __restrict__ y,
                          AT omega) {
  dep_enter();
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)rows * N) return;
  jacobi0_elem<N, AT, TD, TC, false>(t, dinv, b, y, omega);
}

// Tentative transfers: restriction b_c[I] = sum of r over I's members
// (ascending), prolongation-correction x[i] += x_c[agg[i]].
template <int N, class AT, class TC, bool COH>
__device__ __forceinline__ void restrict_elem(size_t t, const int32_t* __restrict__ mptr,
                                              const int32_t* __restrict__ mem, const TC* r, TC* bc) {
  const size_t I = t / N;
  const int c = (int)(t - I * N);
  AT acc = 0;
  for (int q = mptr[I]; q < mptr[I + 1]; ++q) {
    if constexpr (COH) acc += (AT)__ldcg(r + (size_t)mem[q] * N + c);
    else acc += (AT)r[(size_t)mem[q] * N + c];
  }
  bc[t] = (TC)acc;
}

template <int N, class AT, class TC>
__global__ void k_restrict_tent(int nagg, const int32_t* __restrict__ mptr, const int32_t* __restrict__ mem,
                                const TC* __restrict__ r, TC* __restrict__ bc) {
  dep_enter();
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)nagg * N) return;
  restrict_elem<N, AT, TC, false>(t, mptr, mem, r, bc);
}

template <int N, class TC, bool COH>
__device__ __forceinline__ void prolong_elem(size_t t, const int32_t* __restrict__ agg, const TC* xc, TC* x) {
  const size_t i = t / N;
  const int c = (int)(t - i * N);
  if constexpr (COH) x[t] = __ldcg(x + t) + __ldcg(xc + (size_t)agg[i] * N + c);
  else x[t] = x[t] + xc[(size_t)agg[i] * N + c];
}

template <int N, class TC>
__global__ void k_prolong_tent(int rows, const int32_t* __restrict__ agg, const TC* __restrict__ xc,
                               TC* __restrict__ x) {
  dep_enter();
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)rows * N) return;
  prolong_elem<N, TC, false>(t, agg, xc, x);
}

// Coarsest level: x = Ainv b with the dense FP64 inverse, warp per row.
template <class TC, bool COH>
__device__ __forceinline__ void gemv_row(int row, int Nc, const double* __restrict__ inv, const TC* b, TC* x) {
  const int lane = threadIdx.x & 31;
  double acc = 0.0;
  for (int c = lane; c < Nc; c += 32) {
    double bc;
    if constexpr (COH) bc = (double)__ldcg(b + c);
    else bc = (double)b[c];
    acc = fma(inv[(size_t)row * Nc + c], bc, acc);
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
  if (lane == 0) x[row] = (TC)acc;
}

template <class TC>
__global__ void k_coarse_gemv(int Nc, const double* __restrict__ inv, const TC* __restrict__ b,
                              TC* __restrict__ x) {
  dep_enter();
  const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (row >= Nc) return;
  gemv_row<TC, false>(row, Nc, inv, b, x);
}

template <class TI, class TO>
__global__ void k_cast(size_t n, const TI* __restrict__ in, TO* __restrict__ out) {
  dep_enter();
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    out[t] = (TO)in[t];
}

__global__ void k_cast_bf16(size_t n, const double* __restrict__ in, bf16* __restrict__ out) {
  dep_enter();
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    out[t] = __double2bfloat16(in[t]);
}

unsigned rows_grid(int rows, int n) {
  const int rpw = 32 / n;
  const size_t warps = ((size_t)rows + rpw - 1) / rpw;
  return grid_for(warps * 32, 128);
}

// ---- coarse tail: the V-cycle below a size threshold in one cluster launch ----
// The levels from lv[tail_level] down are small enough that a launch per
// sweep, residual and transfer is mostly launch latency. Their part of the
// cycle runs instead as one launch of a thread-block cluster (8 or 16 SMs):
// a list of phases, the same operations in the same order as the kernel by
// kernel cycle launches (Cycle::run), with a cluster barrier between phases.
// Every element is computed by the same device function as in the separate
// kernels, so the results are identical bit for bit; vectors written by
// earlier phases are read through L2 (ld.global.cg), which the cluster
// barrier's release / acquire makes coherent across the cluster's SMs.
namespace cg = cooperative_groups;

constexpr int TAIL_THREADS = 512;

template <int N, class TV>
__global__ void __launch_bounds__(TAIL_THREADS) k_tail(const TailPhase* __restrict__ ph, int nph,
                                                      const TailLevel* __restrict__ lvl, float* const* __restrict__ vec,
                                                      const float* root_b, float* root_x, const double* __restrict__ cinv,
                                                      int cN, float omega) {
  dep_enter();
  cg::cluster_group cl = cg::this_cluster();
  const int nthr = (int)(cl.num_blocks() * blockDim.x);
  const int g = (int)(cl.block_rank() * blockDim.x + threadIdx.x);
  const int gw = g >> 5, nw = nthr >> 5;
  auto V = [&](int id) -> float* {
    return id < 0 ? nullptr : id == 0 ? const_cast<float*>(root_b) : id == 1 ? root_x : vec[id];
  };
  for (int p = 0; p < nph; ++p) {
    const TailPhase f = ph[p];
    const TailLevel& L = lvl[f.level];
    const float* a = V(f.ia);
    const float* b = V(f.ib);
    float* y = V(f.iy);
    switch (f.op) {
      case T_JAC0:
        for (size_t t = g; t < (size_t)L.rows * N; t += nthr)
          jacobi0_elem<N, float, float, float, true>(t, L.dinv, b, y, omega);
        break;
      case T_SWEEP:
        for (int sl = gw; sl < L.nslices; sl += nw)
          sell_slice<N, TV, true, true>(sl, L.rows, L.rp, L.sptr, L.sci, (const TV*)L.sv, L.dinv, a, b, y, omega);
        break;
      case T_RESID:
        for (int sl = gw; sl < L.nslices; sl += nw)
          sell_slice<N, TV, false, true>(sl, L.rows, L.rp, L.sptr, L.sci, (const TV*)L.sv, nullptr, a, b, y, 0.f);
        break;
      case T_RESTRICT:
        for (size_t t = g; t < (size_t)L.nagg * N; t += nthr)
          restrict_elem<N, float, float, true>(t, L.mptr, L.mem, a, y);
        break;
      case T_PROLONG:
        for (size_t t = g; t < (size_t)L.rows * N; t += nthr) prolong_elem<N, float, true>(t, L.agg, a, y);
        break;
      case T_GEMV:
        for (int row = gw; row < cN; row += nw) gemv_row<float, true>(row, cN, cinv, b, y);
        break;
      default:  // T_ZERO
        for (size_t t = g; t < (size_t)L.rows * N; t += nthr) y[t] = 0.f;
        break;
    }
    cl.sync();
  }
}

// ---- one-launch DILU smoothing step for small levels --------------------------
// A level below a size threshold runs a whole DILU / SGS step as one launch
// of a thread-block cluster: the residual r = b - A x (when the level has the
// lane-per-row layout; otherwise it is launched before), then the forward
// sweep colour by colour and the backward sweep in reverse colour order, with
// a cluster barrier between phases. Each row is computed by the same device
// functions as the per-colour launches (identical results); vectors written
// by earlier phases are read through L2, which the barrier's release /
// acquire makes coherent across the cluster's SMs.
constexpr int DC_THREADS = 512;

struct DiluClusterArgs {
  int rows, nslices, ncol;
  const int32_t *rp, *sptr, *sci;  // lane-per-row sliced copy (the residual)
  const void* sv;
  const int32_t *cstart, *crow, *dptr, *dmid, *dci;
  const void* dval;  // split-order values
  const float* einv;
  const float* b;
  float *x, *r, *y, *d;
};

template <int N, class TV, bool RESID>
__global__ void __launch_bounds__(DC_THREADS) k_dilu_cluster(const DiluClusterArgs A) {
  dep_enter();
  cg::cluster_group cl = cg::this_cluster();
  const int g = (int)(cl.block_rank() * blockDim.x + threadIdx.x);
  const int gw = g >> 5, nw = (int)(cl.num_blocks() * blockDim.x) >> 5;
  constexpr int RPW = 32 / N;
  const int lane = threadIdx.x & 31, rw = lane / N, r = lane - rw * N;
  if constexpr (RESID) {
    for (int sl = gw; sl < A.nslices; sl += nw)
      sell_slice<N, TV, false, true>(sl, A.rows, A.rp, A.sptr, A.sci, (const TV*)A.sv, nullptr, A.x, A.b, A.r, 0.f);
    cl.sync();
  }
  const TV* dv = (const TV*)A.dval;
  for (int c = 0; c < A.ncol; ++c) {
    const int t0 = __ldg(A.cstart + c), cnt = __ldg(A.cstart + c + 1) - t0;
    for (int base = gw * RPW; base < cnt; base += nw * RPW) {  // uniform across the warp
      const int mi = base + rw;
      const bool active = rw < RPW && mi < cnt;
      const int t = t0 + (active ? mi : 0);
      const int i = active ? __ldg(A.crow + t) : 0;
      dilu_row<N, float, TV, float, float, true, false, true>(active, i, t, rw, r, A.dptr, A.dmid, nullptr, A.dci,
                                                               dv, A.einv, A.r, A.y, A.d, A.x);
    }
    cl.sync();
  }
  for (int c = A.ncol - 1; c >= 0; --c) {
    const int t0 = __ldg(A.cstart + c), cnt = __ldg(A.cstart + c + 1) - t0;
    for (int base = gw * RPW; base < cnt; base += nw * RPW) {
      const int mi = base + rw;
      const bool active = rw < RPW && mi < cnt;
      const int t = t0 + (active ? mi : 0);
      const int i = active ? __ldg(A.crow + t) : 0;
      dilu_row<N, float, TV, float, float, false, false, true>(active, i, t, rw, r, A.dptr, A.dmid, nullptr, A.dci,
                                                                dv, A.einv, A.r, A.y, A.d, A.x);
    }
    if (c > 0) cl.sync();
  }
}

// ---- batched V-cycle: blockIdx.z selects the case ------------------------------
// One launch per phase of each level covers every case that has that level
// (and whose FGMRES step is live); each element is computed by the device
// function of the single-system kernel in the level's own layout, so every
// case gets the bits of its own cycle. Vector roles: 0 vb, 1 vx, 2 vr, 3 vt.
__device__ __forceinline__ const BLevel* b_level(const BCase& c, int level, int coarse) {
  if (level >= c.n_levels || !*c.live) return nullptr;
  const BLevel* L = &c.lv[level];
  if (coarse ? L->coarse_kind != 1 : L->coarse_kind >= 0) return nullptr;
  return L;
}

__device__ __forceinline__ float* b_vec(const BLevel& L, int role) {
  return role == 0 ? L.vb : role == 1 ? L.vx : role == 2 ? L.vr : L.vt;
}

template <int N, class TV, bool JACOBI>
__global__ void __launch_bounds__(128) kb_sweep_k(const BCase* __restrict__ cases, int level, int coarse, int ix,
                                                  int iy, float omega) {
  dep_enter();
  const BLevel* L = b_level(cases[blockIdx.z], level, coarse);
  if (!L) return;
  const int sl = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (sl >= L->nslices) return;
  const float* x = b_vec(*L, ix);
  float* y = b_vec(*L, iy);
  if (L->smap == 1)
    tpr_slice<N, TV, JACOBI>(sl, L->rows, L->rp, L->srow, L->sptr, L->sci, (const TV*)L->sv, L->dinv, x, L->vb, y,
                             omega);
  else
    sell_slice<N, TV, JACOBI, false>(sl, L->rows, L->rp, L->sptr, L->sci, (const TV*)L->sv, L->dinv, x, L->vb, y,
                                     omega);
}

template <int N>
__global__ void kb_jac0_k(const BCase* __restrict__ cases, int level, int coarse, int iy, float omega) {
  dep_enter();
  const BLevel* L = b_level(cases[blockIdx.z], level, coarse);
  if (!L) return;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t < (size_t)L->rows * N) jacobi0_elem<N, float, float, float, false>(t, L->dinv, L->vb, b_vec(*L, iy), omega);
}

template <int N>
__global__ void kb_zero_k(const BCase* __restrict__ cases, int level, int iy) {
  dep_enter();
  const BLevel* L = b_level(cases[blockIdx.z], level, 0);
  if (!L) return;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t < (size_t)L->rows * N) b_vec(*L, iy)[t] = 0.f;
}

template <int N>
__global__ void kb_restrict_k(const BCase* __restrict__ cases, int level) {
  dep_enter();
  const BCase& c = cases[blockIdx.z];
  const BLevel* L = b_level(c, level, 0);
  if (!L) return;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t < (size_t)L->nagg * N) restrict_elem<N, float, float, false>(t, L->mptr, L->mem, L->vr, c.lv[level + 1].vb);
}

template <int N>
__global__ void kb_prolong_k(const BCase* __restrict__ cases, int level, int iy) {
  dep_enter();
  const BCase& c = cases[blockIdx.z];
  const BLevel* L = b_level(c, level, 0);
  if (!L) return;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t < (size_t)L->rows * N) prolong_elem<N, float, false>(t, L->agg, c.lv[level + 1].vx, b_vec(*L, iy));
}

__global__ void kb_gemv_k(const BCase* __restrict__ cases) {
  dep_enter();
  const BCase& c = cases[blockIdx.z];
  if (!*c.live) return;
  const BLevel& L = c.lv[c.n_levels - 1];
  if (L.coarse_kind != 0) return;
  const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (row < c.cN) gemv_row<float, false>(row, c.cN, c.cinv, L.vb, L.vx);
}

// w = A kt (live cases) / r = b - A x (cases of the round), FP64
template <int N>
__global__ void __launch_bounds__(128) kb_spmv_w_k(const BCase* __restrict__ cases) {
  dep_enter();
  const BCase& c = cases[blockIdx.z];
  if (!*c.live) return;
  RowMap<N> m(c.rows);
  if (m.active) rows_eval<N, double, double, double, double, M_SPMV>(m.i, m.r, c.rp, c.ci, c.val, c.kt, c.w, nullptr);
}

template <int N>
__global__ void __launch_bounds__(128) kb_resid_r_k(const BCase* __restrict__ cases) {
  dep_enter();
  const BCase& c = cases[blockIdx.z];
  if (!*c.round) return;
  RowMap<N> m(c.rows);
  if (m.active) rows_eval<N, double, double, double, double, M_RESID>(m.i, m.r, c.rp, c.ci, c.val, c.x, c.r, c.b);
}

}  // namespace

template <class TI, class TO>
bcs_status cast_vec(Solver* s, const TI* in, TO* out, size_t N) {
  unsigned g = grid_for(N, 256);
  if (g > 148u * 16u) g = 148u * 16u;
  if constexpr (std::is_same<TO, bf16>::value) {
    BCS_LAUNCH_DEP(s, K_CAST, (double)N * (sizeof(TI) + sizeof(TO)), 0, k_cast_bf16, g, 256, 0, N, in, out);
  } else {
    BCS_LAUNCH_DEP(s, K_CAST, (double)N * (sizeof(TI) + sizeof(TO)), 0, (k_cast<TI, TO>), g, 256, 0, N, in, out);
  }
  return BCS_OK;
}
template bcs_status cast_vec<double, float>(Solver*, const double*, float*, size_t);
template bcs_status cast_vec<float, double>(Solver*, const float*, double*, size_t);
template bcs_status cast_vec<double, double>(Solver*, const double*, double*, size_t);
template bcs_status cast_vec<double, bf16>(Solver*, const double*, bf16*, size_t);

bool cycle_is_float(const Solver* s) {
  return (s->setup_cfg.precond == BCS_PC_AMG || s->setup_cfg.precond == BCS_PC_SGS) &&
         s->setup_cfg.precision != BCS_PREC_FP64;
}

// ------------------------------------------------------------ outer FP64 SpMV
bcs_status spmv64(Solver* s, const Bsr& A, const void* x, bool x_is_float, double* y, const double* b,
                  int kind) {
  const int rows = A.rows;
  return with_n(s->n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    const double bytes = (double)A.nnz * (N * N * 8 + 4) + 4.0 * (rows + 1) +
                         (double)rows * N * ((x_is_float ? 4 : 8) + 8 + (b ? 8 : 0));
    const double flops = 2.0 * A.nnz * N * N;
    const unsigned g = rows_grid(rows, N);
    if (x_is_float) {
      if (b)
        BCS_LAUNCH_DEP(s, kind, bytes, flops, (k_rows<N, double, double, float, double, M_RESID>), g, 128, 0, rows,
                   A.rp.p, A.ci.p, A.v.p, (const float*)x, y, b);
      else
        BCS_LAUNCH_DEP(s, kind, bytes, flops, (k_rows<N, double, double, float, double, M_SPMV>), g, 128, 0, rows,
                   A.rp.p, A.ci.p, A.v.p, (const float*)x, y, b);
    } else {
      if (b)
        BCS_LAUNCH_DEP(s, kind, bytes, flops, (k_rows<N, double, double, double, double, M_RESID>), g, 128, 0, rows,
                   A.rp.p, A.ci.p, A.v.p, (const double*)x, y, b);
      else
        BCS_LAUNCH_DEP(s, kind, bytes, flops, (k_rows<N, double, double, double, double, M_SPMV>), g, 128, 0, rows,
                   A.rp.p, A.ci.p, A.v.p, (const double*)x, y, b);
    }
    return BCS_OK;
  });
}

// ------------------------------------------------------------------- V-cycle
namespace {

// Typed views of a cycle with matrix storage TV, inverse storage TD, vector
// type TC and accumulator AT.
template <class TV, class TD, class TC, class AT>
struct Cycle {
  Solver* s;
  static const TV* mat(const Level& L);
  static const TD* dinv(const Level& L);
  static const TV* pmat(const Level& L);
  static const TV* rmat(const Level& L);
  static const TV* smat(const Level& L);

  template <int N>
  bcs_status sweep0(const Level& L, const TC* b, TC* y) {
    const int rows = L.A.rows;
    const AT om = (AT)s->setup_cfg.jacobi_omega;
    BCS_LAUNCH_DEP(s, K_SWEEP, (double)rows * N * (N * sizeof(TD) + 2 * sizeof(TC)), 2.0 * rows * N * N,
               (k_jacobi0<N, AT, TD, TC>), grid_for((size_t)rows * N, 256), 256, 0, rows, dinv(L), b, y, om);
    return BCS_OK;
  }
  template <int N>
  bcs_status sweep(const Level& L, const TC* x, const TC* b, TC* y) {
    const int rows = L.A.rows;
    const AT om = (AT)s->setup_cfg.jacobi_omega;
    const double bytes = (double)L.A.nnz * (N * N * sizeof(TV) + 4) + 4.0 * (rows + 1) +
                         (double)rows * N * (N * sizeof(TD) + 3 * sizeof(TC));
    if constexpr (std::is_same<TC, float>::value) {
      if (L.smap == 1)
        BCS_LAUNCH_DEP(s, K_SWEEP, bytes, 2.0 * (L.A.nnz + rows) * N * N, (k_tpr<N, TV, true>),
                   grid_for((size_t)L.nslices * 32, 128), 128, 0, rows, L.nslices, L.A.rp.p, L.srow.p, L.sptr.p,
                   L.sci.p,
                   smat(L), dinv(L), x, b, y, om);
      else
        BCS_LAUNCH_DEP(s, K_SWEEP, bytes, 2.0 * (L.A.nnz + rows) * N * N, (k_sell<N, TV, true>),
                   grid_for((size_t)L.nslices * 32, 128), 128, 0, rows, L.nslices, L.A.rp.p, L.sptr.p, L.sci.p,
                   smat(L), dinv(L), x, b, y, om);
    } else {
      BCS_LAUNCH_DEP(s, K_SWEEP, bytes, 2.0 * (L.A.nnz + rows) * N * N, (k_jacobi<N, AT, TV, TD, TC>),
                 rows_grid(rows, N), 128, 0, rows, L.A.rp.p, L.A.ci.p, mat(L), dinv(L), x, b, y, om);
    }
    return BCS_OK;
  }
  template <int N>
  bcs_status resid(const Level& L, const TC* x, const TC* b, TC* r) {
    const int rows = L.A.rows;
    const double bytes = (double)L.A.nnz * (N * N * sizeof(TV) + 4) + 4.0 * (rows + 1) +
                         (double)rows * N * 3 * sizeof(TC);
    if constexpr (std::is_same<TC, float>::value) {
      if (L.smap == 1)
        BCS_LAUNCH_DEP(s, K_RESID, bytes, 2.0 * L.A.nnz * N * N, (k_tpr<N, TV, false>),
                   grid_for((size_t)L.nslices * 32, 128), 128, 0, rows, L.nslices, L.A.rp.p, L.srow.p, L.sptr.p,
                   L.sci.p,
                   smat(L), (const float*)nullptr, x, b, r, 0.f);
      else
        BCS_LAUNCH_DEP(s, K_RESID, bytes, 2.0 * L.A.nnz * N * N, (k_sell<N, TV, false>),
                   grid_for((size_t)L.nslices * 32, 128), 128, 0, rows, L.nslices, L.A.rp.p, L.sptr.p, L.sci.p,
                   smat(L), (const float*)nullptr, x, b, r, 0.f);
    } else {
      BCS_LAUNCH_DEP(s, K_RESID, bytes, 2.0 * L.A.nnz * N * N, (k_rows<N, AT, TV, TC, TC, M_RESID>),
                 rows_grid(rows, N), 128, 0, rows, L.A.rp.p, L.A.ci.p, mat(L), x, r, b);
    }
    return BCS_OK;
  }
  static const TV* dmat(const Level& L);
  static const TD* deinv(const Level& L);

  // One DILU step x <- x + M^{-1} (b - A x).
  template <int N>
  bcs_status dilu_step(const Level& L, TC* x, const TC* b) {
    TC* r = (TC*)L.vr.p;
    TC* y = (TC*)L.vt.p;
    TC* d = (TC*)L.vd.p;
    if constexpr (std::is_same<TC, float>::value) {
      if (L.dcl > 0) {
        // the whole step as one cluster launch (the residual inside it when
        // the level has the lane-per-row layout)
        const bool inner = L.smap == 0;
        if (!inner) BCS_OKR(resid<N>(L, x, b, r));
        const DiluClusterArgs A{L.A.rows, L.nslices, L.ncol, L.A.rp.p, L.sptr.p, L.sci.p, smat(L),
                                L.cstart_d.p, L.crow.p, L.dptr.p, L.dmid.p, L.dci.p, dmat(L), deinv(L),
                                (const float*)b, (float*)x, (float*)r, (float*)y, (float*)d};
        cudaLaunchConfig_t lc{};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = L.dcl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        lc.gridDim = dim3(L.dcl);
        lc.blockDim = dim3(DC_THREADS);
        lc.dynamicSmemBytes = 0;
        lc.stream = s->stream;
        lc.attrs = at;
        lc.numAttrs = 1;
        const double per_row = (double)N * N * sizeof(TV) + N * N * sizeof(TD) + 3.0 * N * sizeof(TC);
        const double rbytes = (double)L.A.nnz * (N * N * sizeof(TV) + 4) + 4.0 * (L.A.rows + 1) +
                              (double)L.A.rows * N * 3 * sizeof(TC);
        s->pre(K_SWEEP);
        if (inner) BCS_CU(s, cudaLaunchKernelEx(&lc, k_dilu_cluster<N, TV, true>, A));
        else BCS_CU(s, cudaLaunchKernelEx(&lc, k_dilu_cluster<N, TV, false>, A));
        return s->post(K_SWEEP, "k_dilu_cluster", 2.0 * per_row * L.A.rows + (inner ? rbytes : 0.0),
                       2.0 * (L.A.nnz + 2.0 * L.A.rows) * N * N);
      }
    }
    BCS_OKR(resid<N>(L, x, b, r));
    constexpr bool G = std::is_same<TV, double>::value;  // FP64: the BSR values through dsrc
    const double per_row = (double)N * N * sizeof(TV) + N * N * sizeof(TD) + 3.0 * N * sizeof(TC);
    for (int c = 0; c < L.ncol; ++c) {
      const int b0 = L.cstart[c], m = L.cstart[c + 1] - b0;
      if (m > 0)
        BCS_LAUNCH_DEP(s, K_SWEEP, per_row * m, 2.0 * m * N * N, (k_dilu_sweep<N, AT, TV, TD, TC, true, G>),
                   rows_grid(m, N), 128, 0, m, b0, L.crow.p, L.dptr.p, L.dmid.p, L.dsrc.p, L.dci.p, dmat(L),
                   deinv(L), r, y, d, x);
    }
    for (int c = L.ncol - 1; c >= 0; --c) {
      const int b0 = L.cstart[c], m = L.cstart[c + 1] - b0;
      if (m > 0)
        BCS_LAUNCH_DEP(s, K_SWEEP, per_row * m, 2.0 * m * N * N, (k_dilu_sweep<N, AT, TV, TD, TC, false, G>),
                   rows_grid(m, N), 128, 0, m, b0, L.crow.p, L.dptr.p, L.dmid.p, L.dsrc.p, L.dci.p, dmat(L),
                   deinv(L), r, y, d, x);
    }
    return BCS_OK;
  }

  template <int N>
  bcs_status restrict_(const Level& L, const TC* r, TC* bc) {
    if (s->setup_cfg.pmode == BCS_P_TENTATIVE) {
      BCS_LAUNCH_DEP(s, K_TRANSFER, (double)(L.A.rows + L.nagg) * N * sizeof(TC) + 4.0 * L.A.rows, 0,
                 (k_restrict_tent<N, AT, TC>), grid_for((size_t)L.nagg * N, 256), 256, 0, L.nagg, L.mptr.p,
                 L.mem.p, r, bc);
    } else {
      const Bsr& R = L.R;
      BCS_LAUNCH_DEP(s, K_TRANSFER, (double)R.nnz * (N * N * sizeof(TV) + 4), 2.0 * R.nnz * N * N,
                 (k_rows<N, AT, TV, TC, TC, M_SPMV>), rows_grid(R.rows, N), 128, 0, R.rows, R.rp.p, R.ci.p,
                 rmat(L), r, bc, (const TC*)nullptr);
    }
    return BCS_OK;
  }
  template <int N>
  bcs_status prolong(const Level& L, const TC* xc, TC* x) {
    if (s->setup_cfg.pmode == BCS_P_TENTATIVE) {
      BCS_LAUNCH_DEP(s, K_TRANSFER, (double)L.A.rows * N * 3 * sizeof(TC) + 4.0 * L.A.rows, 0,
                 (k_prolong_tent<N, TC>), grid_for((size_t)L.A.rows * N, 256), 256, 0, L.A.rows, L.agg.p, xc, x);
    } else {
      const Bsr& P = L.P;
      BCS_LAUNCH_DEP(s, K_TRANSFER, (double)P.nnz * (N * N * sizeof(TV) + 4), 2.0 * P.nnz * N * N,
                 (k_rows<N, AT, TV, TC, TC, M_ADD>), rows_grid(P.rows, N), 128, 0, P.rows, P.rp.p, P.ci.p,
                 pmat(L), xc, x, (const TC*)nullptr);
    }
    return BCS_OK;
  }

  // count >= 1 sweeps from zero; the start buffer is chosen so the last
  // sweep lands in x.
  template <int N>
  bcs_status sweeps_from_zero(const Level& L, int count, const TC* b, TC* x, TC* tmp) {
    TC* cur = ((count - 1) % 2 == 0) ? x : tmp;
    TC* alt = cur == x ? tmp : x;
    BCS_OKR(sweep0<N>(L, b, cur));
    for (int k = 1; k < count; ++k) {
      BCS_OKR(sweep<N>(L, cur, b, alt));
      std::swap(cur, alt);
    }
    return BCS_OK;
  }

  // Stand-alone SGS preconditioner on level 0: x = M^-1 b, the smoother step
  // from x = 0 (block Jacobi when the level has more than 128 colours).
  template <int N>
  bcs_status sgs(const TC* b, TC* x) {
    Level& L = s->lv[0];
    const int rows = L.A.rows;
    if (L.ncol > 0) {
      BCS_CU(s, cudaMemsetAsync(x, 0, (size_t)rows * N * sizeof(TC), s->stream));
      return dilu_step<N>(L, x, b);
    }
    BCS_LAUNCH_DEP(s, K_SWEEP, (double)rows * N * (N * sizeof(TD) + 2 * sizeof(TC)), 2.0 * rows * N * N,
               (k_jacobi0<N, AT, TD, TC>), grid_for((size_t)rows * N, 256), 256, 0, rows, dinv(L), b, x, (AT)1);
    return BCS_OK;
  }
  // the levels from s->tail_level down as one cluster launch
  template <int N>
  bcs_status tail(const float* b, float* x) {
    const TailPlan& T = s->tail;
    cudaLaunchConfig_t lc{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = T.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.gridDim = dim3(T.cluster);
    lc.blockDim = dim3(TAIL_THREADS);
    lc.dynamicSmemBytes = 0;
    lc.stream = s->stream;
    lc.attrs = at;
    lc.numAttrs = 1;
    const TailPhase* ph = (const TailPhase*)T.buf.p;
    const TailLevel* lvl = (const TailLevel*)(T.buf.p + T.level_off);
    float* const* vec = (float* const*)(T.buf.p + T.vec_off);
    s->pre(K_SWEEP);
    BCS_CU(s, cudaLaunchKernelEx(&lc, k_tail<N, TV>, ph, T.nph, lvl, vec, b, x, (const double*)s->cinv.p, s->cN,
                                 (float)s->setup_cfg.jacobi_omega));
    return s->post(K_SWEEP, "k_tail", T.bytes, T.flops);
  }

  template <int N>
  bcs_status run(int l, const TC* b, TC* x) {
    LevelScope level_scope(s, l);
    if constexpr (std::is_same<TC, float>::value)
      if (l == s->tail_level) return tail<N>((const float*)b, (float*)x);
    Level& L = s->lv[l];
    const int nu1 = s->setup_cfg.nu1, nu2 = s->setup_cfg.nu2;
    TC* tmp = (TC*)L.vt.p;
    if (L.coarse_kind == 0) {
      BCS_LAUNCH_DEP(s, K_COARSE, 8.0 * s->cN * s->cN, 2.0 * s->cN * s->cN, k_coarse_gemv<TC>,
                 grid_for((size_t)s->cN * 32, 256), 256, 0, s->cN, s->cinv.p, b, x);
      return BCS_OK;
    }
    if (L.ncol > 0) {
      // DILU: every step, the first included, is the general step from x = 0
      BCS_CU(s, cudaMemsetAsync(x, 0, (size_t)L.A.rows * N * sizeof(TC), s->stream));
      if (L.coarse_kind == 1) {
        for (int k = 0; k < s->setup_cfg.coarse_sweeps; ++k) BCS_OKR(dilu_step<N>(L, x, b));
        return BCS_OK;
      }
      for (int k = 0; k < nu1; ++k) BCS_OKR(dilu_step<N>(L, x, b));
      Level& Lc = s->lv[l + 1];
      TC* r = (TC*)L.vr.p;
      BCS_OKR(resid<N>(L, x, b, r));
      BCS_OKR(restrict_<N>(L, r, (TC*)Lc.vb.p));
      BCS_OKR(run<N>(l + 1, (const TC*)Lc.vb.p, (TC*)Lc.vx.p));
      BCS_OKR(prolong<N>(L, (const TC*)Lc.vx.p, x));
      for (int k = 0; k < nu2; ++k) BCS_OKR(dilu_step<N>(L, x, b));
      return BCS_OK;
    }
    if (L.coarse_kind == 1) return sweeps_from_zero<N>(L, s->setup_cfg.coarse_sweeps, b, x, tmp);
    const int swaps = (nu1 > 1 ? nu1 - 1 : 0) + nu2;
    TC* cur = swaps % 2 == 0 ? x : tmp;
    TC* alt = cur == x ? tmp : x;
    if (nu1 >= 1) {
      BCS_OKR(sweep0<N>(L, b, cur));
      for (int k = 1; k < nu1; ++k) {
        BCS_OKR(sweep<N>(L, cur, b, alt));
        std::swap(cur, alt);
      }
    } else {
      BCS_CU(s, cudaMemsetAsync(cur, 0, (size_t)L.A.rows * N * sizeof(TC), s->stream));
    }
    Level& Lc = s->lv[l + 1];
    TC* r = (TC*)L.vr.p;
    BCS_OKR(resid<N>(L, cur, b, r));
    BCS_OKR(restrict_<N>(L, r, (TC*)Lc.vb.p));
    BCS_OKR(run<N>(l + 1, (const TC*)Lc.vb.p, (TC*)Lc.vx.p));
    BCS_OKR(prolong<N>(L, (const TC*)Lc.vx.p, cur));
    for (int k = 0; k < nu2; ++k) {
      BCS_OKR(sweep<N>(L, cur, b, alt));
      std::swap(cur, alt);
    }
    return BCS_OK;
  }
};

template <> const double* Cycle<double, double, double, double>::dmat(const Level& L) { return L.A.v.p; }
template <> const double* Cycle<double, double, double, double>::deinv(const Level& L) { return L.einv.p; }
template <> const float* Cycle<float, float, float, float>::dmat(const Level& L) { return L.a32.p; }
template <> const float* Cycle<float, float, float, float>::deinv(const Level& L) { return L.einv32.p; }
template <> const bf16* Cycle<bf16, float, float, float>::dmat(const Level& L) { return L.a16.p; }
template <> const float* Cycle<bf16, float, float, float>::deinv(const Level& L) { return L.einv32.p; }
template <> const double* Cycle<double, double, double, double>::mat(const Level& L) { return L.A.v.p; }
template <> const double* Cycle<double, double, double, double>::dinv(const Level& L) { return L.dinv.p; }
template <> const double* Cycle<double, double, double, double>::pmat(const Level& L) { return L.P.v.p; }
template <> const double* Cycle<double, double, double, double>::rmat(const Level& L) { return L.R.v.p; }
template <> const double* Cycle<double, double, double, double>::smat(const Level&) { return nullptr; }
template <> const float* Cycle<float, float, float, float>::smat(const Level& L) { return L.s32.p; }
template <> const bf16* Cycle<bf16, float, float, float>::smat(const Level& L) { return L.s16.p; }
template <> const float* Cycle<float, float, float, float>::mat(const Level&) { return nullptr; }
template <> const float* Cycle<float, float, float, float>::dinv(const Level& L) { return L.dinv32.p; }
template <> const float* Cycle<float, float, float, float>::pmat(const Level& L) { return L.P32.p; }
template <> const float* Cycle<float, float, float, float>::rmat(const Level& L) { return L.R32.p; }
template <> const bf16* Cycle<bf16, float, float, float>::mat(const Level&) { return nullptr; }
template <> const float* Cycle<bf16, float, float, float>::dinv(const Level& L) { return L.dinv32.p; }
template <> const bf16* Cycle<bf16, float, float, float>::pmat(const Level& L) { return L.P16.p; }
template <> const bf16* Cycle<bf16, float, float, float>::rmat(const Level& L) { return L.R16.p; }

template <class TV, class TD, class TC, class AT>
bcs_status run_cycle(Solver* s, const TC* b, TC* x) {
  Cycle<TV, TD, TC, AT> c{s};
  return with_n(s->n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    return c.template run<N>(0, b, x);
  });
}

}  // namespace

// Sliced copy of level L's operator in layout `map` and the cycle precision
// (structure once per hierarchy and layout, values at every setup / resetup).
// Structure of layout `map` for level L (slice order and lengths, their
// scan): launched only; the step count is copied to *steps_dev for the
// caller to read. False in *needed when L already has that structure.
bcs_status layout_structure(Solver* s, Level& L, int map, int32_t* steps_dev, bool* needed) {
  const int n = s->n, rows = L.A.rows, rpw = map == 1 ? 32 : 32 / n;
  *needed = L.nslices == 0 || L.smap != map;
  if (!*needed) return BCS_OK;
  if (!s->lv.empty() && &L == &s->lv[0]) s->v0_direct = -1;  // a copy in the old layout
  L.tpos.release();
  L.sci.release();
  L.s32.release();
  L.s16.release();
  L.srow.release();
  const int ns = (rows + rpw - 1) / rpw;
  DBuf<int32_t> slen;
  BCS_ALLOC(s, slen, ns);
  BCS_ALLOC(s, L.sptr, ns + 1);
  if (map == 1) {
    BCS_ALLOC(s, L.srow, rows);
    BCS_LAUNCH_DEP(s, K_CAST, 0, 0, k_window_order, grid_for(rows, SORT_WIN), SORT_WIN, 0, rows, L.A.rp.p, L.srow.p);
  }
  BCS_LAUNCH_DEP(s, K_CAST, 0, 0, k_slice_len, grid_for(ns, 256), 256, 0, rows, rpw, ns, L.A.rp.p, L.srow.p, slen.p);
  BCS_OKR(exclusive_scan(s, slen.p, L.sptr.p, ns));
  BCS_CU(s, cudaMemcpyAsync(steps_dev, L.sptr.p + ns, sizeof(int32_t), cudaMemcpyDeviceToDevice, s->stream));
  L.nslices = ns;
  L.smap = map;
  return BCS_OK;
}

// Values of level L's sliced copy (its structure in place, nsteps known).
bcs_status layout_values(Solver* s, Level& L, int prec) {
  const int n = s->n, rows = L.A.rows, map = L.smap, rpw = map == 1 ? 32 : 32 / n;
  if (&L == &s->lv[0] && s->v0_direct >= 0) {
    const bool written = s->v0_direct == prec && map == 1 && L.tpos.p && L.sci.p;
    s->v0_direct = -1;
    if (written) return BCS_OK;  // the value gather wrote this copy
  }
  if (!L.sci.p) BCS_ALLOC(s, L.sci, (size_t)L.nsteps * rpw);
  const size_t nv = (size_t)L.nsteps * rpw * n * n;
  // the fine level's first fill in layout 1 also records the slot map
  // (slots in int32)
  int32_t* tpos = nullptr;
  if (map == 1 && &L == &s->lv[0] && !L.tpos.p && (size_t)L.nsteps * 32 <= (size_t)INT32_MAX) {
    BCS_ALLOC(s, L.tpos, L.A.nnz > 0 ? L.A.nnz : 1);
    tpos = L.tpos.p;
  }
  return with_n(n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    const unsigned g = grid_for((size_t)L.nslices * 32, 128);
    const double bytes = (double)L.A.nnz * N * N * (8 + (prec == BCS_PREC_FP32 ? 4 : 2));
    if (prec == BCS_PREC_FP32) {
      BCS_ALLOC(s, L.s32, nv);
      if (map == 1)
        BCS_LAUNCH_DEP(s, K_CAST, bytes, 0, (k_tpr_fill<N, float>), g, 128, 0, rows, L.nslices, L.A.rp.p, L.A.ci.p,
                   L.A.v.p, L.srow.p, L.sptr.p, L.sci.p, L.s32.p, tpos);
      else
        BCS_LAUNCH_DEP(s, K_CAST, bytes, 0, (k_slice_fill<N, float>), g, 128, 0, rows, L.nslices, L.A.rp.p,
                   L.A.ci.p, L.A.v.p, L.sptr.p, L.sci.p, L.s32.p);
    } else {
      BCS_ALLOC(s, L.s16, nv);
      if (map == 1)
        BCS_LAUNCH_DEP(s, K_CAST, bytes, 0, (k_tpr_fill<N, bf16>), g, 128, 0, rows, L.nslices, L.A.rp.p, L.A.ci.p,
                   L.A.v.p, L.srow.p, L.sptr.p, L.sci.p, L.s16.p, tpos);
      else
        BCS_LAUNCH_DEP(s, K_CAST, bytes, 0, (k_slice_fill<N, bf16>), g, 128, 0, rows, L.nslices, L.A.rp.p,
                   L.A.ci.p, L.A.v.p, L.sptr.p, L.sci.p, L.s16.p);
    }
    return BCS_OK;
  });
}

// Sliced copy of level L in layout `map` (structure when new, values).
bcs_status fill_layout(Solver* s, Level& L, int prec, int map) {
  DBuf<int32_t> steps;
  BCS_ALLOC(s, steps, 1);
  bool needed = false;
  BCS_OKR(layout_structure(s, L, map, steps.p, &needed));
  if (needed) {
    int32_t h = 0;
    BCS_CU(s, cudaMemcpyAsync(&h, steps.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
    BCS_CU(s, cudaStreamSynchronize(s->stream));
    L.nsteps = h;
  }
  return layout_values(s, L, prec);
}

// ---- layout autotuner --------------------------------------------------------
// For a level of at least TUNE_MIN_ROWS block rows, both layouts are built and
// one smoother sweep of each is timed (CUDA events, best of TUNE_REPS after a
// warm-up launch); the faster layout is kept. Decisions are cached per
// process by (n, precision, log2 rows, blocks per row x 4), so later setups of
// similar levels skip the timing. Both layouts give identical results.
constexpr int TUNE_MIN_ROWS = 4096;
constexpr int TUNE_REPS = 3;

std::mutex g_tune_mu;
std::map<std::array<int, 4>, int> g_tune_cache;

template <int N, class TV>
bcs_status time_sweep(Solver* s, const Level& L, cudaEvent_t e0, cudaEvent_t e1, float* best) {
  const TV* sv;
  if constexpr (std::is_same<TV, bf16>::value) sv = L.s16.p;
  else sv = L.s32.p;
  const float* x = (const float*)L.vx.p;
  const float* b = (const float*)L.vb.p;
  float* y = (float*)L.vt.p;
  const unsigned g = grid_for((size_t)L.nslices * 32, 128);
  *best = 1e30f;
  for (int rep = 0; rep <= TUNE_REPS; ++rep) {
    BCS_CU(s, cudaEventRecord(e0, s->stream));
    if (L.smap == 1)
      BCS_LAUNCH(s, K_TUNE, 0, 0, (k_tpr<N, TV, true>), g, 128, 0, L.A.rows, L.nslices, L.A.rp.p, L.srow.p,
                 L.sptr.p, L.sci.p, sv, L.dinv32.p, x, b, y, 0.8f);
    else
      BCS_LAUNCH(s, K_TUNE, 0, 0, (k_sell<N, TV, true>), g, 128, 0, L.A.rows, L.nslices, L.A.rp.p, L.sptr.p,
                 L.sci.p, sv, L.dinv32.p, x, b, y, 0.8f);
    BCS_CU(s, cudaEventRecord(e1, s->stream));
    BCS_CU(s, cudaEventSynchronize(e1));
    float ms = 0.f;
    BCS_CU(s, cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0 && ms < *best) *best = ms;
  }
  return BCS_OK;
}

bcs_status choose_layout(Solver* s, Level& L, int prec, int* map) {
  *map = 0;
  const int rows = L.A.rows;
  if (rows < TUNE_MIN_ROWS) return BCS_OK;
  int lg = 0;
  while ((1 << (lg + 1)) <= rows) ++lg;
  const std::array<int, 4> key{s->n, prec, lg, (int)(4.0 * L.A.nnz / rows + 0.5)};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      *map = it->second;
      return BCS_OK;
    }
  }
  const size_t N = (size_t)rows * s->n;
  BCS_CU(s, cudaMemsetAsync(L.vx.p, 0, N * sizeof(float), s->stream));
  BCS_CU(s, cudaMemsetAsync(L.vb.p, 0, N * sizeof(float), s->stream));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BCS_CU(s, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return s->fail(BCS_ECUDA, "cudaEventCreate failed");
  }
  float t[2] = {0.f, 0.f};
  bcs_status st = BCS_OK;
  for (int m = 0; m < 2 && st == BCS_OK; ++m) {
    st = fill_layout(s, L, prec, m);
    if (st == BCS_OK)
      st = with_n(s->n, [&](auto NC) -> bcs_status {
        constexpr int NN = decltype(NC)::value;
        return prec == BCS_PREC_FP32 ? time_sweep<NN, float>(s, L, e0, e1, &t[m])
                                     : time_sweep<NN, bf16>(s, L, e0, e1, &t[m]);
      });
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  BCS_OKR(st);
  *map = t[1] < t[0] ? 1 : 0;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = *map;
  return BCS_OK;
}

// Layout of level L's sliced copy: kept, forced by the configuration, or
// picked by the autotuner (which builds and times both).
bcs_status slice_map(Solver* s, Level& L, int prec, bool tail, int* map) {
  *map = L.smap;
  if (tail) *map = 0;  // the coarse-tail kernel walks the lane-per-row layout
  if (*map < 0) {
    if (s->setup_cfg.slice_layout >= 0) *map = s->setup_cfg.slice_layout;
    else BCS_OKR(choose_layout(s, L, prec, map));
  }
  return BCS_OK;
}

// Blocks of the one-launch DILU step's cluster on this device: 16 (a
// non-portable size) when a cluster that large can be resident, else 8, else
// 0 (per-colour launches).
template <int N, class TV>
int dilu_cluster_blocks() {
  for (int cs : {16, 8}) {
    if (cs > 8 &&
        (cudaFuncSetAttribute(k_dilu_cluster<N, TV, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
             cudaSuccess ||
         cudaFuncSetAttribute(k_dilu_cluster<N, TV, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
             cudaSuccess)) {
      (void)cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t lc{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.gridDim = dim3(cs);
    lc.blockDim = dim3(DC_THREADS);
    lc.attrs = at;
    lc.numAttrs = 1;
    int n1 = 0, n2 = 0;
    if (cudaOccupancyMaxActiveClusters(&n1, k_dilu_cluster<N, TV, true>, &lc) == cudaSuccess &&
        cudaOccupancyMaxActiveClusters(&n2, k_dilu_cluster<N, TV, false>, &lc) == cudaSuccess && n1 >= 1 &&
        n2 >= 1)
      return cs;
    (void)cudaGetLastError();
  }
  return 0;
}

// Cycle vectors and storage copies of the hierarchy in the configured
// precision (after every setup / resetup).
// ---- coarse-tail plan ----------------------------------------------------------
namespace {

// The phases Cycle::run would launch for the levels from lt down, in order,
// with the same buffer choices (vector ids: 0 / 1 the tail's b / x; per tail
// level 2 + 4 (l - lt) + {vb, vx, vr, vt}).
struct TailGen {
  Solver* s;
  int lt;
  std::vector<TailPhase> ph;
  double bytes = 0.0, flops = 0.0;
  int id(int l, int k) const { return 2 + 4 * (l - lt) + k; }
  void push(int op, int l, int ia, int ib, int iy) { ph.push_back(TailPhase{op, l - lt, ia, ib, iy}); }
  void account(int op, const Level& L) {
    const double n = s->n, nn = n * n, rows = L.A.rows, nnz = L.A.nnz;
    const double vb = s->setup_cfg.precision == BCS_PREC_FP32 ? 4.0 : 2.0;
    switch (op) {
      case T_SWEEP: bytes += nnz * (nn * vb + 4) + 4 * (rows + 1) + rows * n * (n * 4 + 12); flops += 2 * (nnz + rows) * nn; break;
      case T_RESID: bytes += nnz * (nn * vb + 4) + 4 * (rows + 1) + rows * n * 12; flops += 2 * nnz * nn; break;
      case T_JAC0: bytes += rows * n * (n * 4 + 8); flops += 2 * rows * nn; break;
      case T_RESTRICT: bytes += (rows + L.nagg) * n * 4 + 4 * rows; break;
      case T_PROLONG: bytes += rows * n * 12 + 4 * rows; break;
      case T_GEMV: bytes += 8.0 * s->cN * s->cN; flops += 2.0 * s->cN * s->cN; break;
      default: bytes += rows * n * 4; break;
    }
  }
  void op(int o, int l, int ia, int ib, int iy) {
    push(o, l, ia, ib, iy);
    account(o, s->lv[l]);
  }
  void gen(int l, int b, int x) {
    const Level& L = s->lv[l];
    const bcs_config& c = s->setup_cfg;
    if (L.coarse_kind == 0) {
      op(T_GEMV, l, -1, b, x);
      return;
    }
    const int tmp = id(l, 3);
    if (L.coarse_kind == 1) {  // Cycle::sweeps_from_zero
      const int count = c.coarse_sweeps;
      int cur = ((count - 1) % 2 == 0) ? x : tmp, alt = cur == x ? tmp : x;
      op(T_JAC0, l, -1, b, cur);
      for (int k = 1; k < count; ++k) {
        op(T_SWEEP, l, cur, b, alt);
        std::swap(cur, alt);
      }
      return;
    }
    const int swaps = (c.nu1 > 1 ? c.nu1 - 1 : 0) + c.nu2;
    int cur = swaps % 2 == 0 ? x : tmp, alt = cur == x ? tmp : x;
    if (c.nu1 >= 1) {
      op(T_JAC0, l, -1, b, cur);
      for (int k = 1; k < c.nu1; ++k) {
        op(T_SWEEP, l, cur, b, alt);
        std::swap(cur, alt);
      }
    } else {
      op(T_ZERO, l, -1, -1, cur);
    }
    const int r = id(l, 2);
    op(T_RESID, l, cur, b, r);
    op(T_RESTRICT, l, r, -1, id(l + 1, 0));
    gen(l + 1, id(l + 1, 0), id(l + 1, 1));
    op(T_PROLONG, l, id(l + 1, 1), -1, cur);
    for (int k = 0; k < c.nu2; ++k) {
      op(T_SWEEP, l, cur, b, alt);
      std::swap(cur, alt);
    }
  }
};

// Largest cluster (16, else 8 SMs) that can be resident for the tail kernel.
template <int N, class TV>
bcs_status tail_cluster(Solver* s, int* cluster) {
  *cluster = 0;
  for (int cs : {16, 8}) {
    if (cs > 8 &&
        cudaFuncSetAttribute(k_tail<N, TV>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      (void)cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t lc{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.gridDim = dim3(cs);
    lc.blockDim = dim3(TAIL_THREADS);
    lc.attrs = at;
    lc.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k_tail<N, TV>, &lc) == cudaSuccess && nc >= 1) {
      *cluster = cs;
      return BCS_OK;
    }
    (void)cudaGetLastError();
  }
  return BCS_OK;
}

}  // namespace

// Phase list, level table and vector table of the coarse tail, in one device
// buffer; the tail is switched off when no cluster of 8 fits.
bcs_status build_tail(Solver* s) {
  const int lt = s->tail_level, nl = (int)s->lv.size();
  int cluster = 0;
  BCS_OKR(with_n(s->n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    return s->setup_cfg.precision == BCS_PREC_FP32 ? tail_cluster<N, float>(s, &cluster)
                                                   : tail_cluster<N, bf16>(s, &cluster);
  }));
  if (cluster == 0) {
    s->tail_level = -1;
    return BCS_OK;
  }
  TailGen gen{s, lt};
  gen.gen(lt, 0, 1);
  std::vector<TailLevel> lvl(nl - lt);
  std::vector<float*> vec(2 + 4 * (nl - lt), nullptr);
  for (int l = lt; l < nl; ++l) {
    const Level& L = s->lv[l];
    TailLevel& t = lvl[l - lt];
    t.rows = L.A.rows;
    t.nslices = L.nslices;
    t.nagg = L.nagg;
    t.pad = 0;
    t.rp = L.A.rp.p;
    t.sptr = L.sptr.p;
    t.sci = L.sci.p;
    t.mptr = L.mptr.p;
    t.mem = L.mem.p;
    t.agg = L.agg.p;
    t.sv = s->setup_cfg.precision == BCS_PREC_FP32 ? (const void*)L.s32.p : (const void*)L.s16.p;
    t.dinv = L.dinv32.p;
    vec[2 + 4 * (l - lt) + 0] = (float*)L.vb.p;
    vec[2 + 4 * (l - lt) + 1] = (float*)L.vx.p;
    vec[2 + 4 * (l - lt) + 2] = (float*)L.vr.p;
    vec[2 + 4 * (l - lt) + 3] = (float*)L.vt.p;
  }
  TailPlan& T = s->tail;
  const size_t a = gen.ph.size() * sizeof(TailPhase);
  T.level_off = (a + 255) / 256 * 256;
  T.vec_off = T.level_off + (lvl.size() * sizeof(TailLevel) + 255) / 256 * 256;
  const size_t total = T.vec_off + vec.size() * sizeof(float*);
  std::vector<char> host(total, 0);
  std::memcpy(host.data(), gen.ph.data(), a);
  std::memcpy(host.data() + T.level_off, lvl.data(), lvl.size() * sizeof(TailLevel));
  std::memcpy(host.data() + T.vec_off, vec.data(), vec.size() * sizeof(float*));
  BCS_ALLOC(s, T.buf, total);
  BCS_CU(s, cudaMemcpyAsync(T.buf.p, host.data(), total, cudaMemcpyHostToDevice, s->stream));
  BCS_CU(s, cudaStreamSynchronize(s->stream));  // the host staging goes out of scope
  T.nph = (int)gen.ph.size();
  T.cluster = cluster;
  T.bytes = gen.bytes;
  T.flops = gen.flops;
  return BCS_OK;
}

bcs_status cycle_prepare(Solver* s, bool keep_graphs) {
  if (!keep_graphs) s->drop_graph();
  const int prec = s->setup_cfg.precision;
  const size_t vsz = prec == BCS_PREC_FP64 ? sizeof(double) : sizeof(float);
  const int n = s->n, nn = n * n;
  const bool sliced = prec != BCS_PREC_FP64 && (s->setup_cfg.precond == BCS_PC_AMG || s->setup_cfg.precond == BCS_PC_SGS);
  const size_t nl = s->lv.size();
  s->tail_level = -1;
  s->tail.nph = 0;
  if (sliced && s->setup_cfg.precond == BCS_PC_AMG && s->setup_cfg.pmode == BCS_P_TENTATIVE &&
      s->setup_cfg.tail_rows > 0 && s->n <= 8) {
    bool dilu = false;
    for (const Level& L : s->lv) dilu |= L.ncol > 0;
    if (!dilu)
      for (size_t l = 0; l < nl; ++l)
        if (s->lv[l].A.rows <= s->setup_cfg.tail_rows) {
          s->tail_level = (int)l;
          break;
        }
  }
  // slice structures of every level first; their step counts are read back
  // together in one round trip
  DBuf<int32_t> steps;
  BCS_ALLOC(s, steps, nl);
  std::vector<char> needed(nl, 0);
  int dcl_blocks = -1;  // cluster size of the one-launch DILU step, looked up once
  for (size_t l = 0; l < nl; ++l) {
    Level& L = s->lv[l];
    LevelScope level_scope(s, (int)l);
    const size_t N = (size_t)L.A.rows * n;
    BCS_ALLOC(s, L.vx, N * vsz);
    BCS_ALLOC(s, L.vb, N * vsz);
    BCS_ALLOC(s, L.vr, N * vsz);
    BCS_ALLOC(s, L.vt, N * vsz);
    if (L.ncol > 0) BCS_ALLOC(s, L.vd, N * vsz);
    L.dcl = 0;
    if (!sliced) continue;
    BCS_OKR(dilu_prepare(s, L));
    if (L.ncol > 0 && L.A.rows <= s->setup_cfg.dilu_cluster_rows) {
      if (dcl_blocks < 0)
        BCS_OKR(with_n(n, [&](auto NC) -> bcs_status {
          constexpr int NB = decltype(NC)::value;
          dcl_blocks = prec == BCS_PREC_FP32 ? dilu_cluster_blocks<NB, float>() : dilu_cluster_blocks<NB, bf16>();
          return BCS_OK;
        }));
      L.dcl = dcl_blocks;
    }
    BCS_ALLOC(s, L.dinv32, (size_t)L.A.rows * nn);
    if (L.dinv64) BCS_OKR(cast_vec<double, float>(s, L.dinv.p, L.dinv32.p, (size_t)L.A.rows * nn));
    int map = 0;
    BCS_OKR(slice_map(s, L, prec, s->tail_level >= 0 && (int)l >= s->tail_level, &map));
    bool need = false;
    BCS_OKR(layout_structure(s, L, map, steps.p + l, &need));
    needed[l] = need;
  }
  if (sliced && std::find(needed.begin(), needed.end(), 1) != needed.end()) {
    std::vector<int32_t> h(nl, 0);
    BCS_CU(s, cudaMemcpyAsync(h.data(), steps.p, nl * sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
    BCS_CU(s, cudaStreamSynchronize(s->stream));
    for (size_t l = 0; l < nl; ++l)
      if (needed[l]) s->lv[l].nsteps = h[l];
  }
  for (size_t l = 0; l < nl && sliced; ++l) {
    Level& L = s->lv[l];
    LevelScope level_scope(s, (int)l);
    BCS_OKR(layout_values(s, L, prec));
    const bool smoothed = L.coarse_kind < 0 && s->setup_cfg.pmode == BCS_P_SMOOTHED;
    if (prec == BCS_PREC_FP32) {
      if (smoothed) {
        BCS_ALLOC(s, L.P32, (size_t)L.P.nnz * nn);
        BCS_ALLOC(s, L.R32, (size_t)L.R.nnz * nn);
        BCS_OKR(cast_vec<double, float>(s, L.P.v.p, L.P32.p, (size_t)L.P.nnz * nn));
        BCS_OKR(cast_vec<double, float>(s, L.R.v.p, L.R32.p, (size_t)L.R.nnz * nn));
      }
    } else if (smoothed) {
      BCS_ALLOC(s, L.P16, (size_t)L.P.nnz * nn);
      BCS_ALLOC(s, L.R16, (size_t)L.R.nnz * nn);
      BCS_OKR(cast_vec<double, bf16>(s, L.P.v.p, L.P16.p, (size_t)L.P.nnz * nn));
      BCS_OKR(cast_vec<double, bf16>(s, L.R.v.p, L.R16.p, (size_t)L.R.nnz * nn));
    }
  }
  if (s->tail_level >= 0) BCS_OKR(build_tail(s));
  return BCS_OK;
}

namespace {
bool sliced_cycle(const bcs_config& c) {
  return c.precision != BCS_PREC_FP64 && (c.precond == BCS_PC_AMG || c.precond == BCS_PC_SGS);
}
}  // namespace

bcs_status fine_slice_target(Solver* s, SliceTarget* t) {
  *t = SliceTarget{};
  if (s->lv.empty()) return BCS_OK;
  // the configuration the next setup takes: the new one for a full setup
  const bcs_config& c = s->have_hierarchy ? s->setup_cfg : s->cfg;
  Level& L = s->lv[0];
  if (!sliced_cycle(c) || L.smap != 1 || !L.tpos.p || !L.sci.p || L.nslices == 0) return BCS_OK;
  if (c.slice_layout == 0 || (c.tail_rows > 0 && L.A.rows <= c.tail_rows)) return BCS_OK;
  const size_t nv = (size_t)L.nsteps * 32 * s->n * s->n;
  if (c.precision == BCS_PREC_FP32 && L.s32.p && L.s32.n == nv) t->s32 = L.s32.p;
  else if (c.precision == BCS_PREC_BF16 && L.s16.p && L.s16.n == nv) t->s16 = L.s16.p;
  else return BCS_OK;
  t->tpos = L.tpos.p;
  t->prec = c.precision;
  return BCS_OK;
}

namespace {

// Kinds of the kernels inside the cycle: with per-launch events on any of
// them the cycle runs kernel by kernel.
constexpr int CYCLE_KINDS = (1 << K_SWEEP) | (1 << K_RESID) | (1 << K_TRANSFER) | (1 << K_COARSE);

bool use_graph(const Solver* s) {
  if (s->setup_cfg.precision == BCS_PREC_FP64 || s->cfg.cycle_graph == 0) return false;
  if (s->cfg.profile && (s->cfg.profile_kinds == 0 || (s->cfg.profile_kinds & CYCLE_KINDS))) return false;
  return true;
}

template <class TV>
bcs_status run_cycle_f(Solver* s, const float* b, float* x) {
  return run_cycle<TV, float, float, float>(s, b, x);
}

// Replays the cycle lv[0].vb -> lv[0].vx as one CUDA graph, capturing it on
// first use after a setup. The captured launches are counted in the solver's
// statistics at every replay, as if launched one by one.
template <class TV>
bcs_status graph_cycle(Solver* s) {
  Level& L0 = s->lv[0];
  if (!s->cyc_exec) {
    long long kl[BCS_NUM_KERNEL_KINDS];
    double kb[BCS_NUM_KERNEL_KINDS], kf[BCS_NUM_KERNEL_KINDS];
    const long long l0 = s->launches;
    for (int k = 0; k < BCS_NUM_KERNEL_KINDS; ++k) {
      kl[k] = s->kind_launches[k];
      kb[k] = s->kind_bytes[k];
      kf[k] = s->kind_flops[k];
    }
    // capture on a private stream (the solver's may be the legacy default
    // stream, which cannot be captured); the graph is then launched on the
    // solver's stream
    if (!s->gstream) BCS_CU(s, cudaStreamCreateWithFlags(&s->gstream, cudaStreamNonBlocking));
    const cudaStream_t own = s->stream;
    BCS_CU(s, cudaStreamBeginCapture(s->gstream, cudaStreamCaptureModeThreadLocal));
    s->stream = s->gstream;
    const bcs_status st = run_cycle_f<TV>(s, (const float*)L0.vb.p, (float*)L0.vx.p);
    s->stream = own;
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s->gstream, &g);
    // the capture ran nothing: take its launches back out of the statistics
    s->launches = l0;
    for (int k = 0; k < BCS_NUM_KERNEL_KINDS; ++k) {
      s->cyc_kind_launches[k] = s->kind_launches[k] - kl[k];
      s->cyc_kind_bytes[k] = s->kind_bytes[k] - kb[k];
      s->cyc_kind_flops[k] = s->kind_flops[k] - kf[k];
      s->kind_launches[k] = kl[k];
      s->kind_bytes[k] = kb[k];
      s->kind_flops[k] = kf[k];
    }
    if (st != BCS_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (ce != cudaSuccess) return s->fail(BCS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    const cudaError_t ie = cudaGraphInstantiate(&s->cyc_exec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      s->cyc_exec = nullptr;
      return s->fail(BCS_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
    }
  }
  BCS_CU(s, cudaGraphLaunch(s->cyc_exec, s->stream));
  for (int k = 0; k < BCS_NUM_KERNEL_KINDS; ++k) {
    s->launches += s->cyc_kind_launches[k];
    s->kind_launches[k] += s->cyc_kind_launches[k];
    s->kind_bytes[k] += s->cyc_kind_bytes[k];
    s->kind_flops[k] += s->cyc_kind_flops[k];
  }
  return BCS_OK;
}

}  // namespace

// z = M^{-1} v in the cycle precision; v is FP64 (a Krylov vector).
bcs_status precond_apply(Solver* s, const double* v, void* z) {
  Level& L0 = s->lv[0];
  const size_t N = (size_t)L0.A.rows * s->n;
  if (s->setup_cfg.precision == BCS_PREC_FP64) return run_cycle<double, double, double, double>(s, v, (double*)z);
  BCS_OKR(cast_vec<double, float>(s, v, (float*)L0.vb.p, N));
  if (!use_graph(s))
    return s->setup_cfg.precision == BCS_PREC_FP32 ? run_cycle_f<float>(s, (const float*)L0.vb.p, (float*)z)
                                                   : run_cycle_f<bf16>(s, (const float*)L0.vb.p, (float*)z);
  BCS_OKR(s->setup_cfg.precision == BCS_PREC_FP32 ? graph_cycle<float>(s) : graph_cycle<bf16>(s));
  BCS_CU(s, cudaMemcpyAsync(z, L0.vx.p, N * sizeof(float), cudaMemcpyDeviceToDevice, s->stream));
  return BCS_OK;
}

template <class TV, class TD, class TC, class AT>
bcs_status run_sgs(Solver* s, const TC* b, TC* x) {
  Cycle<TV, TD, TC, AT> c{s};
  return with_n(s->n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    return c.template sgs<N>(b, x);
  });
}

// z = M^-1 v for the stand-alone SGS preconditioner, in the cycle precision.
bcs_status sgs_apply(Solver* s, const double* v, void* z) {
  Level& L0 = s->lv[0];
  const size_t N = (size_t)L0.A.rows * s->n;
  const int prec = s->setup_cfg.precision;
  if (prec == BCS_PREC_FP64) return run_sgs<double, double, double, double>(s, v, (double*)z);
  BCS_OKR(cast_vec<double, float>(s, v, (float*)L0.vb.p, N));
  return prec == BCS_PREC_FP32 ? run_sgs<float, float, float, float>(s, (const float*)L0.vb.p, (float*)z)
                               : run_sgs<bf16, float, float, float>(s, (const float*)L0.vb.p, (float*)z);
}

bcs_status precond_cycle64(Solver* s, const double* v, double* z) {
  return run_cycle<double, double, double, double>(s, v, z);
}

bcs_status precond_cycle32(Solver* s, const float* v, float* z) {
  return s->setup_cfg.precision == BCS_PREC_FP32 ? run_cycle_f<float>(s, v, z) : run_cycle_f<bf16>(s, v, z);
}

bcs_status sgs_fixed(Solver* s, const void* v, void* z) {
  const int prec = s->setup_cfg.precision;
  if (prec == BCS_PREC_FP64) return run_sgs<double, double, double, double>(s, (const double*)v, (double*)z);
  return prec == BCS_PREC_FP32 ? run_sgs<float, float, float, float>(s, (const float*)v, (float*)z)
                               : run_sgs<bf16, float, float, float>(s, (const float*)v, (float*)z);
}

// Block-Jacobi preconditioner (one undamped block solve): z = D^-1 v.
bcs_status jacobi_apply(Solver* s, const double* v, double* z) {
  Level& L0 = s->lv[0];
  return with_n(s->n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    const int rows = L0.A.rows;
    BCS_LAUNCH_DEP(s, K_SWEEP, (double)rows * N * (N * 8 + 16), 2.0 * rows * N * N, (k_jacobi0<N, double, double, double>),
               grid_for((size_t)rows * N, 256), 256, 0, rows, L0.dinv.p, v, z, 1.0);
    return BCS_OK;
  });
}


// ---- batched V-cycle and products (host side) ----------------------------------
namespace {

template <int N, class TV>
bcs_status kb_cycle_t(Solver* s, const BCase* cases, const std::vector<BCase>& host, int count) {
  const bcs_config& c = s->setup_cfg;
  const float om = (float)c.jacobi_omega;
  int lmax = 0;
  for (const BCase& h : host) lmax = std::max(lmax, h.n_levels);
  // largest work of level l over the cases
  auto most = [&](int l, auto f) {
    size_t m = 0;
    for (const BCase& h : host)
      if (l < h.n_levels) m = std::max<size_t>(m, f(h.lv[l]));
    return m;
  };
  auto slices = [&](int l) { return grid_for(most(l, [](const BLevel& L) { return (size_t)L.nslices; }) * 32, 128); };
  auto elems = [&](int l) { return grid_for(most(l, [](const BLevel& L) { return (size_t)L.rows * N; }), 256); };
  const dim3 z1(1, 1, count);
  auto grid = [&](unsigned g) { return dim3(g, 1, count); };
  const int swaps = (c.nu1 > 1 ? c.nu1 - 1 : 0) + c.nu2;
  const int cur0 = swaps % 2 == 0 ? 1 : 3, alt0 = cur0 == 1 ? 3 : 1;
  int cur_down = cur0, alt_down = alt0;
  for (int k = 1; k < c.nu1; ++k) std::swap(cur_down, alt_down);
  // down: pre-smoothing, residual, restriction
  for (int l = 0; l + 1 < lmax; ++l) {
    int cur = cur0, alt = alt0;
    if (c.nu1 >= 1) {
      BCS_LAUNCH_DEP(s, K_SWEEP, 0, 0, (kb_jac0_k<N>), grid(elems(l)), 256, 0, cases, l, 0, cur, om);
      for (int k = 1; k < c.nu1; ++k) {
        BCS_LAUNCH_DEP(s, K_SWEEP, 0, 0, (kb_sweep_k<N, TV, true>), grid(slices(l)), 128, 0, cases, l, 0, cur, alt, om);
        std::swap(cur, alt);
      }
    } else {
      BCS_LAUNCH_DEP(s, K_SWEEP, 0, 0, (kb_zero_k<N>), grid(elems(l)), 256, 0, cases, l, cur);
    }
    BCS_LAUNCH_DEP(s, K_RESID, 0, 0, (kb_sweep_k<N, TV, false>), grid(slices(l)), 128, 0, cases, l, 0, cur, 2, 0.f);
    const unsigned ga = grid_for(most(l, [](const BLevel& L) { return (size_t)L.nagg * N; }), 256);
    BCS_LAUNCH_DEP(s, K_TRANSFER, 0, 0, (kb_restrict_k<N>), grid(ga), 256, 0, cases, l);
  }
  // coarsest levels: dense inverses, or smoother sweeps from zero
  int cn = 0;
  for (const BCase& h : host) cn = std::max(cn, h.cN);
  if (cn > 0) BCS_LAUNCH_DEP(s, K_COARSE, 0, 0, kb_gemv_k, grid(grid_for((size_t)cn * 32, 256)), 256, 0, cases);
  for (int l = 0; l < lmax; ++l) {
    bool any = false;
    for (const BCase& h : host) any |= l < h.n_levels && h.lv[l].coarse_kind == 1;
    if (!any) continue;
    const int n_sw = c.coarse_sweeps;
    int cur = ((n_sw - 1) % 2 == 0) ? 1 : 3, alt = cur == 1 ? 3 : 1;
    BCS_LAUNCH_DEP(s, K_SWEEP, 0, 0, (kb_jac0_k<N>), grid(elems(l)), 256, 0, cases, l, 1, cur, om);
    for (int k = 1; k < n_sw; ++k) {
      BCS_LAUNCH_DEP(s, K_SWEEP, 0, 0, (kb_sweep_k<N, TV, true>), grid(slices(l)), 128, 0, cases, l, 1, cur, alt, om);
      std::swap(cur, alt);
    }
  }
  // up: prolongation-correction, post-smoothing
  for (int l = lmax - 2; l >= 0; --l) {
    int cur = cur_down, alt = alt_down;
    BCS_LAUNCH_DEP(s, K_TRANSFER, 0, 0, (kb_prolong_k<N>), grid(elems(l)), 256, 0, cases, l, cur);
    for (int k = 0; k < c.nu2; ++k) {
      BCS_LAUNCH_DEP(s, K_SWEEP, 0, 0, (kb_sweep_k<N, TV, true>), grid(slices(l)), 128, 0, cases, l, 0, cur, alt, om);
      std::swap(cur, alt);
    }
  }
  (void)z1;
  return BCS_OK;
}

}  // namespace

bcs_status kb_cycle(Solver* s, const BCase* cases, const std::vector<BCase>& host, int count) {
  return with_n(s->n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    return s->setup_cfg.precision == BCS_PREC_FP32 ? kb_cycle_t<N, float>(s, cases, host, count)
                                                   : kb_cycle_t<N, bf16>(s, cases, host, count);
  });
}

bcs_status kb_spmv_w(Solver* s, const BCase* cases, int count, int max_rows) {
  return with_n(s->n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    BCS_LAUNCH_DEP(s, K_SPMV64, 0, 0, kb_spmv_w_k<N>, dim3(rows_grid(max_rows, N), 1, count), 128, 0, cases);
    return BCS_OK;
  });
}

bcs_status kb_resid_r(Solver* s, const BCase* cases, int count, int max_rows) {
  return with_n(s->n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    BCS_LAUNCH_DEP(s, K_SPMV64, 0, 0, kb_resid_r_k<N>, dim3(rows_grid(max_rows, N), 1, count), 128, 0, cases);
    return BCS_OK;
  });
}

}  // namespace bcs
