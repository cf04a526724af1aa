// Multicolour block DILU smoother (Sec. 4: the smoother of the paper's GPU
// runs): colouring, colour-ordered FP64 factorisation, and the forward /
// backward sweeps of one smoothing step x <- x + M^{-1} (b - A x) with
// M = (E + L) E^{-1} (E + U), L / U the blocks A_ij whose column's colour is
// lower / higher than the row's.
//
// Colouring: synchronous Jones-Plassmann rounds. A row's priority is
// (h(i), i), h the 32-bit lowbias32 integer hash (xorshift-multiply rounds
// with the constants 0x7feb352d and 0x846ca68b). In a round every uncoloured
// row whose priority exceeds that of all its uncoloured neighbours takes the
// smallest colour not held by a neighbour coloured in an earlier round.
// Rounds read the previous round's colours only, so the result does not
// depend on scheduling. At most 128 colours; a level that would need more
// keeps block Jacobi.
//
// Factor: E_i = A_ii - sum over j with colour(j) < colour(i) and A_ij != 0,
// columns ascending, of (A_ij E_j^{-1}) A_ji, each block product an fma chain
// from +0 (m ascending); E_i^{-1} by the register Gauss-Jordan of the block
// inverses. Rows of one colour are independent: per colour one launch forms
// E_i, a second inverts it (the Gauss-Jordan's registers kept out of the
// accumulation pass).
#include <algorithm>

#include "gj.cuh"
#include "internal.h"

namespace bcs {

namespace {

constexpr int DILU_MAX_COLOURS = 128;

__device__ __forceinline__ uint32_t lowbias32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// One Jones-Plassmann round: cin -> cout; uncoloured rows after the round are
// counted into *left (one atomic per warp); err |= 32 when a row would need a
// colour >= 128.
__global__ void k_jp_round(int rows, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const int32_t* __restrict__ cin, int32_t* __restrict__ cout, int32_t* __restrict__ left,
                           int32_t* __restrict__ err) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int uncoloured = 0;
  if (i < rows) {
    int c = cin[i];
    if (c < 0) {
      const uint32_t hi = lowbias32((uint32_t)i);
      bool top = true;
      unsigned long long m0 = 0, m1 = 0;
      for (int k = rp[i]; k < rp[i + 1]; ++k) {
        const int j = ci[k];
        if (j == i) continue;
        const int cj = cin[j];
        if (cj < 0) {
          const uint32_t hj = lowbias32((uint32_t)j);
          if (hj > hi || (hj == hi && j > i)) top = false;
        } else if (cj < 64) {
          m0 |= 1ull << cj;
        } else {
          m1 |= 1ull << (cj - 64);
        }
      }
      if (top) {
        if (~m0) c = __ffsll((long long)~m0) - 1;
        else if (~m1) c = 64 + __ffsll((long long)~m1) - 1;
        else atomicOr(err, 32);
      }
      uncoloured = c < 0;
    }
    cout[i] = c;
  }
  const int u = __reduce_add_sync(0xffffffffu, uncoloured);
  if ((threadIdx.x & 31) == 0 && u) atomicAdd(left, u);
}

// Per-colour row counts (block-local histogram, one atomic per colour and
// block). blockDim >= DILU_MAX_COLOURS.
__global__ void k_colour_count(int rows, const int32_t* __restrict__ colour, int32_t* __restrict__ cnt) {
  dep_enter();
  __shared__ int32_t hist[DILU_MAX_COLOURS];
  const int t = threadIdx.x, i = blockIdx.x * blockDim.x + t;
  if (t < DILU_MAX_COLOURS) hist[t] = 0;
  __syncthreads();
  if (i < rows) atomicAdd(&hist[colour[i]], 1);
  __syncthreads();
  if (t < DILU_MAX_COLOURS && hist[t]) atomicAdd(&cnt[t], hist[t]);
}

// Rows grouped by colour: each block reserves one range per colour; the
// order inside a colour does not matter (its rows are independent).
__global__ void k_colour_place(int rows, const int32_t* __restrict__ colour, const int32_t* __restrict__ start,
                               int32_t* __restrict__ cursor, int32_t* __restrict__ crow) {
  dep_enter();
  __shared__ int32_t hist[DILU_MAX_COLOURS], base[DILU_MAX_COLOURS];
  const int t = threadIdx.x, i = blockIdx.x * blockDim.x + t;
  if (t < DILU_MAX_COLOURS) hist[t] = 0;
  __syncthreads();
  const int c = i < rows ? colour[i] : 0;
  const int rank = i < rows ? atomicAdd(&hist[c], 1) : 0;
  __syncthreads();
  if (t < DILU_MAX_COLOURS && hist[t]) base[t] = atomicAdd(&cursor[t], hist[t]);
  __syncthreads();
  if (i < rows) crow[start[c] + base[c] + rank] = i;
}

// Split lists in colour-list order: slot t holds row crow[t], so the rows
// one colour's sweep walks have their lists side by side.
// Off-diagonal blocks of the slot's row whose column has another colour (the
// blocks the sweeps use; a valid colouring leaves only the diagonal out).
__global__ void k_dilu_split_count(int rows, const int32_t* __restrict__ crow, const int32_t* __restrict__ rp,
                                   const int32_t* __restrict__ ci, const int32_t* __restrict__ colour,
                                   int32_t* __restrict__ cnt) {
  dep_enter();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows) return;
  const int i = crow[t], c = colour[i];
  int m = 0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) m += colour[ci[k]] != c;
  cnt[t] = m;
}

// The slot's lower part then its upper part, each in column order.
__global__ void k_dilu_split_fill(int rows, const int32_t* __restrict__ crow, const int32_t* __restrict__ rp,
                                  const int32_t* __restrict__ ci, const int32_t* __restrict__ colour,
                                  const int32_t* __restrict__ dptr, int32_t* __restrict__ dmid,
                                  int32_t* __restrict__ dsrc, int32_t* __restrict__ dci) {
  dep_enter();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows) return;
  const int i = crow[t], c = colour[i];
  int o = dptr[t];
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    const int j = ci[k];
    if (colour[j] < c) {
      dsrc[o] = k;
      dci[o] = j;
      ++o;
    }
  }
  dmid[t] = o;
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    const int j = ci[k];
    if (colour[j] > c) {
      dsrc[o] = k;
      dci[o] = j;
      ++o;
    }
  }
}

// Values of the split blocks in the cycle precision: out[q] = A[dsrc[q]]
// for q < *total (one thread per entry).
template <int NN, class TO>
__global__ void k_dilu_split_values(long long bound, const int32_t* __restrict__ total,
                                    const int32_t* __restrict__ dsrc, const double* __restrict__ val,
                                    TO* __restrict__ out) {
  dep_enter();
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= bound) return;
  const long long q = t / NN;
  if (q >= *total) return;
  const int e = (int)(t - q * NN);
  const double v = val[(size_t)__ldg(dsrc + q) * NN + e];
  if constexpr (std::is_same<TO, bf16>::value) out[t] = __double2bfloat16(v);
  else out[t] = (TO)v;
}

__device__ __forceinline__ int find_pos(const int32_t* __restrict__ ci, int b, int e, int col) {
  while (b < e) {
    const int m = (b + e) >> 1;
    const int cm = ci[m];
    if (cm == col) return m;
    if (cm < col) b = m + 1;
    else e = m;
  }
  return -1;
}

// E_i for the rows of colour c, written to E[q] (q = index in the colour's
// list). n*n <= 32: one warp per row, lane (r, cc) holds E_i[r][cc]; per
// earlier neighbour j it forms W[r][cc] = (A_ij E_j^{-1})[r][cc] and, from
// its row's W by shuffles, Z[r][cc] = (W A_ji)[r][cc], each the fma chain of
// the definition. Larger blocks: one thread per row, W one row at a time.
// T: the arithmetic (double: the factor the oracle reproduces; float: the
// FP32 / BF16 cycle's factor); TA: the type of the blocks read (the FP64
// values, or for T = float an FP32 copy rounded once, so that no conversion
// from FP64 runs per use on the FP64 pipe).
template <int N, class T, class TA>
__global__ void __launch_bounds__(128) k_dilu_schur(int cnt, const int32_t* __restrict__ rows_c, int c,
                                                    const int32_t* __restrict__ colour, const int32_t* __restrict__ rp,
                                                    const int32_t* __restrict__ ci, const TA* __restrict__ val,
                                                    const int32_t* __restrict__ dpos, const T* __restrict__ einv,
                                                    T* __restrict__ E, int32_t* __restrict__ err) {
  dep_enter();
  constexpr int NN = N * N;
  if constexpr (NN <= 32) {
    const int lane = threadIdx.x & 31;
    const int q = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (q >= cnt) return;  // uniform across the warp
    const int i = rows_c[q];
    const bool act = lane < NN;
    const int r = act ? lane / N : 0, cc = act ? lane - (lane / N) * N : 0;
    T m = act ? (T)val[(size_t)dpos[i] * NN + lane] : (T)0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      const int j = ci[k];
      if (colour[j] >= c) continue;
      const int kt = find_pos(ci, rp[j], rp[j + 1], i);
      if (kt < 0) {
        if (lane == 0) atomicOr(err, 128);  // structurally unsymmetric pattern
        return;
      }
      const TA* aij = val + (size_t)k * NN;
      const T* ej = einv + (size_t)j * NN;
      const TA* aji = val + (size_t)kt * NN;
      T w = 0;
#pragma unroll
      for (int mm = 0; mm < N; ++mm) w = fma((T)aij[r * N + mm], ej[mm * N + cc], w);
      T z = 0;
#pragma unroll
      for (int mm = 0; mm < N; ++mm) {
        const T wm = __shfl_sync(0xffffffffu, w, (r * N + mm) & 31);
        z = fma(wm, (T)aji[mm * N + cc], z);
      }
      m = m - z;
    }
    if (act) E[(size_t)q * NN + lane] = m;
  } else {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cnt) return;
    const int i = rows_c[q];
    T M[NN];
    const TA* d = val + (size_t)dpos[i] * NN;
#pragma unroll
    for (int e = 0; e < NN; ++e) M[e] = (T)d[e];
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      const int j = ci[k];
      if (colour[j] >= c) continue;
      const int kt = find_pos(ci, rp[j], rp[j + 1], i);
      if (kt < 0) {
        atomicOr(err, 128);
        return;
      }
      const TA* aij = val + (size_t)k * NN;
      const T* ej = einv + (size_t)j * NN;
      const TA* aji = val + (size_t)kt * NN;
#pragma unroll
      for (int r = 0; r < N; ++r) {
        T w[N];
#pragma unroll
        for (int cc = 0; cc < N; ++cc) {
          T acc = 0;
#pragma unroll
          for (int mm = 0; mm < N; ++mm) acc = fma((T)aij[r * N + mm], ej[mm * N + cc], acc);
          w[cc] = acc;
        }
#pragma unroll
        for (int cc = 0; cc < N; ++cc) {
          T z = 0;
#pragma unroll
          for (int mm = 0; mm < N; ++mm) z = fma(w[mm], (T)aji[mm * N + cc], z);
          M[r * N + cc] = M[r * N + cc] - z;
        }
      }
    }
    T* o = E + (size_t)q * NN;
#pragma unroll
    for (int e = 0; e < NN; ++e) o[e] = M[e];
  }
}

// E_i^{-1} for the rows of colour c from E (one thread per row).
template <int N, class T>
__global__ void __launch_bounds__(64) k_dilu_invert(int cnt, const int32_t* __restrict__ rows_c,
                                                    const T* __restrict__ E, T* __restrict__ einv,
                                                    int32_t* __restrict__ err) {
  dep_enter();
  constexpr int NN = N * N;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= cnt) return;
  BlockGJ<N, T> g;
  const T* a = E + (size_t)q * NN;
#pragma unroll
  for (int r = 0; r < N; ++r)
#pragma unroll
    for (int cc = 0; cc < N; ++cc) g.M[r][cc] = a[r * N + cc];
  if (!gj_finish<N>(g, einv + (size_t)rows_c[q] * NN)) atomicOr(err, 64);
}

// The DILU factor of level L colour by colour (E_i from the Schur sums over
// earlier colours, then E_i^{-1}) into einv, in arithmetic T; reads the
// status flags once at the end.
template <class T>
bcs_status dilu_factor(Solver* s, const Level& L, T* einv) {
  const int n = s->n;
  int maxc = 0;
  for (int c = 0; c < L.ncol; ++c) maxc = std::max(maxc, L.cstart[c + 1] - L.cstart[c]);
  DBuf<T> E;
  BCS_ALLOC(s, E, (size_t)maxc * n * n);
  // the blocks in the arithmetic's type (an FP32 copy for T = float)
  DBuf<T> a_copy;
  const T* va = nullptr;
  if constexpr (std::is_same<T, double>::value) {
    va = L.A.v.p;
  } else {
    BCS_ALLOC(s, a_copy, (size_t)L.A.nnz * n * n);
    BCS_OKR(cast_vec<double, T>(s, L.A.v.p, a_copy.p, (size_t)L.A.nnz * n * n));
    va = a_copy.p;
  }
  BCS_OKR(with_n(n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    for (int c = 0; c < L.ncol; ++c) {
      const int b = L.cstart[c], m = L.cstart[c + 1] - b;
      if (m <= 0) continue;
      const unsigned gs = N * N <= 32 ? grid_for((size_t)m * 32, 128) : grid_for(m, 128);
      BCS_LAUNCH_DEP(s, K_SETUP_INV, sizeof(T) * m * N * N * 4.0, 4.0 * m * N * N * N * 3, (k_dilu_schur<N, T, T>),
                     gs, 128, 0, m, L.crow.p + b, c, L.colour.p, L.A.rp.p, L.A.ci.p, va, L.dpos.p, einv, E.p,
                     s->flag.p);
      BCS_LAUNCH_DEP(s, K_SETUP_INV, 2.0 * sizeof(T) * m * N * N, 4.0 * m * N * N * N, (k_dilu_invert<N, T>),
                     grid_for(m, 64), 64, 0, m, L.crow.p + b, E.p, einv, s->flag.p);
    }
    return BCS_OK;
  }));
  int32_t h = 0;
  BCS_CU(s, cudaMemcpyAsync(&h, s->flag.p, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  if (h & 128) return s->fail(BCS_EINVAL, "DILU needs a structurally symmetric pattern");
  if (h & 64) return s->fail(BCS_SINGULAR_BLOCK, "singular DILU diagonal block");
  return BCS_OK;
}

}  // namespace

bcs_status dilu_setup(Solver* s, Level& L, bool full, bool sgs) {
  const int rows = L.A.rows, n = s->n;
  if (full) {
    L.ncol = -1;
    L.cstart.clear();
    L.colour.release();
    L.crow.release();
    DBuf<int32_t> other, aux;
    BCS_ALLOC(s, L.colour, rows);
    BCS_ALLOC(s, other, rows);
    BCS_ALLOC(s, aux, 2);
    BCS_CU(s, cudaMemsetAsync(L.colour.p, 0xff, rows * sizeof(int32_t), s->stream));
    BCS_CU(s, cudaMemsetAsync(aux.p + 1, 0, sizeof(int32_t), s->stream));
    int32_t* cin = L.colour.p;
    int32_t* cout = other.p;
    int32_t h[2] = {1, 0};
    // Rounds in batches of four between host checks; a round with nothing
    // left to colour copies the colours unchanged.
    for (int round = 0; h[0] > 0 && !(h[1] & 32); ++round) {
      if (round > rows + 4) return s->fail(BCS_EINVAL, "colouring did not finish");
      BCS_CU(s, cudaMemsetAsync(aux.p, 0, sizeof(int32_t), s->stream));
      BCS_LAUNCH_DEP(s, K_SETUP_AGG, 0, 0, k_jp_round, grid_for(rows, 256), 256, 0, rows, L.A.rp.p, L.A.ci.p, cin,
                 cout, aux.p, aux.p + 1);
      std::swap(cin, cout);
      if (round % 4 == 3) {
        BCS_CU(s, cudaMemcpyAsync(h, aux.p, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
        BCS_CU(s, cudaStreamSynchronize(s->stream));
      }
    }
    if (h[1] & 32) return BCS_OK;  // more than 128 colours: this level keeps block Jacobi
    if (cin != L.colour.p) L.colour = std::move(other);
    // colour lists
    DBuf<int32_t> cnt, cursor;
    DBuf<int32_t>& start = L.cstart_d;
    BCS_ALLOC(s, cnt, DILU_MAX_COLOURS);
    BCS_ALLOC(s, start, DILU_MAX_COLOURS + 1);
    BCS_ALLOC(s, cursor, DILU_MAX_COLOURS);
    BCS_CU(s, cudaMemsetAsync(cnt.p, 0, DILU_MAX_COLOURS * sizeof(int32_t), s->stream));
    BCS_CU(s, cudaMemsetAsync(cursor.p, 0, DILU_MAX_COLOURS * sizeof(int32_t), s->stream));
    BCS_LAUNCH_DEP(s, K_SETUP_AGG, 0, 0, k_colour_count, grid_for(rows, 256), 256, 0, rows, L.colour.p, cnt.p);
    std::vector<int32_t> hc(DILU_MAX_COLOURS);
    BCS_CU(s, cudaMemcpyAsync(hc.data(), cnt.p, DILU_MAX_COLOURS * sizeof(int32_t), cudaMemcpyDeviceToHost,
                              s->stream));
    BCS_CU(s, cudaStreamSynchronize(s->stream));
    int ncol = 0;
    for (int c = 0; c < DILU_MAX_COLOURS; ++c)
      if (hc[c] > 0) ncol = c + 1;
    L.cstart.assign(ncol + 1, 0);
    for (int c = 0; c < ncol; ++c) L.cstart[c + 1] = L.cstart[c] + hc[c];
    BCS_CU(s, cudaMemcpyAsync(start.p, L.cstart.data(), (ncol + 1) * sizeof(int32_t), cudaMemcpyHostToDevice,
                              s->stream));
    BCS_ALLOC(s, L.crow, rows);
    BCS_LAUNCH_DEP(s, K_SETUP_AGG, 0, 0, k_colour_place, grid_for(rows, 256), 256, 0, rows, L.colour.p, start.p,
               cursor.p, L.crow.p);
    // the sweeps' split rows (sized by the nonzero count, an upper bound)
    BCS_ALLOC(s, L.dptr, rows + 1);
    BCS_ALLOC(s, L.dmid, rows);
    BCS_ALLOC(s, L.dsrc, L.A.nnz);
    BCS_ALLOC(s, L.dci, L.A.nnz);
    DBuf<int32_t> dcnt;
    BCS_ALLOC(s, dcnt, rows);
    BCS_LAUNCH_DEP(s, K_SETUP_AGG, 0, 0, k_dilu_split_count, grid_for(rows, 256), 256, 0, rows, L.crow.p, L.A.rp.p,
               L.A.ci.p, L.colour.p, dcnt.p);
    BCS_OKR(exclusive_scan(s, dcnt.p, L.dptr.p, rows));
    BCS_LAUNCH_DEP(s, K_SETUP_AGG, 0, 0, k_dilu_split_fill, grid_for(rows, 256), 256, 0, rows, L.crow.p, L.A.rp.p,
               L.A.ci.p, L.colour.p, L.dptr.p, L.dmid.p, L.dsrc.p, L.dci.p);
    // the host vector L.cstart is read by this copy: finish it before return
    BCS_CU(s, cudaStreamSynchronize(s->stream));
    L.ncol = ncol;
  }
  if (L.ncol <= 0) return BCS_OK;
  L.einv64 = true;
  if (sgs) {
    // symmetric Gauss-Seidel: E = D, so E^-1 is the block-Jacobi inverse (the
    // FP32 one when the setup inverted the blocks in FP32 only)
    if (!L.dinv64) {
      L.einv64 = false;
      BCS_ALLOC(s, L.einv32, (size_t)rows * n * n);
      BCS_CU(s, cudaMemcpyAsync(L.einv32.p, L.dinv32.p, (size_t)rows * n * n * sizeof(float),
                                cudaMemcpyDeviceToDevice, s->stream));
      return BCS_OK;
    }
    BCS_ALLOC(s, L.einv, (size_t)rows * n * n);
    BCS_CU(s, cudaMemcpyAsync(L.einv.p, L.dinv.p, (size_t)rows * n * n * sizeof(double), cudaMemcpyDeviceToDevice,
                              s->stream));
    return BCS_OK;
  }
  if (s->setup_cfg.precision == BCS_PREC_FP64) BCS_ALLOC(s, L.einv, (size_t)rows * n * n);
  if (s->setup_cfg.precision != BCS_PREC_FP64) {
    // the FP32 / BF16 cycle's factor, computed in FP32 straight into einv32
    L.einv64 = false;
    BCS_ALLOC(s, L.einv32, (size_t)rows * n * n);
    return dilu_factor<float>(s, L, L.einv32.p);
  }
  return dilu_factor<double>(s, L, L.einv.p);
}

bcs_status dilu_einv64(Solver* s, int l, const double** out, DBuf<double>& tmp) {
  Level& L = s->lv[l];
  if (L.einv64) {
    *out = L.einv.p;
    return BCS_OK;
  }
  const bcs_config& c = s->setup_cfg;
  if (c.precond == BCS_PC_SGS || c.smoother == BCS_SMOOTH_SGS) return level_dinv64(s, l, out, tmp);  // E = D
  BCS_ALLOC(s, tmp, (size_t)L.A.rows * s->n * s->n);
  BCS_OKR(dilu_factor<double>(s, L, tmp.p));
  *out = tmp.p;
  return BCS_OK;
}

bcs_status dilu_prepare(Solver* s, Level& L) {
  if (L.ncol <= 0) return BCS_OK;
  const size_t nn = (size_t)s->n * s->n;
  BCS_ALLOC(s, L.einv32, (size_t)L.A.rows * nn);
  if (L.einv64) BCS_OKR(cast_vec<double, float>(s, L.einv.p, L.einv32.p, (size_t)L.A.rows * nn));
  const long long bound = (long long)L.A.nnz * (long long)nn;
  const bool b16 = s->setup_cfg.precision == BCS_PREC_BF16;
  if (b16) BCS_ALLOC(s, L.a16, (size_t)bound);
  else BCS_ALLOC(s, L.a32, (size_t)bound);
  return with_n(s->n, [&](auto NC) -> bcs_status {
    constexpr int N = decltype(NC)::value;
    const unsigned g = grid_for((size_t)bound, 256);
    if (b16)
      BCS_LAUNCH_DEP(s, K_CAST, 10.0 * bound, 0, (k_dilu_split_values<N * N, bf16>), g, 256, 0, bound,
                 L.dptr.p + L.A.rows, L.dsrc.p, L.A.v.p, L.a16.p);
    else
      BCS_LAUNCH_DEP(s, K_CAST, 12.0 * bound, 0, (k_dilu_split_values<N * N, float>), g, 256, 0, bound,
                 L.dptr.p + L.A.rows, L.dsrc.p, L.A.v.p, L.a32.p);
    return BCS_OK;
  });
}

}  // namespace bcs
