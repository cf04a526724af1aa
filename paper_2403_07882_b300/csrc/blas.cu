// FP64 vector kernels of the Krylov solvers: deterministic multi-dot
// products (a fixed grid and a fixed reduction tree, so results do not depend
// on timing), classical Gram-Schmidt updates, and the axpy family.
#include "internal.h"

namespace bcs {

namespace {

constexpr int RED_BLOCKS = 1184;  // 8 x 148 SMs; fixed, so results do not depend on timing
constexpr int RED_THREADS = 256;
constexpr int MD_CHUNK = 8;      // vectors per multidot block row

// partial[q * RED_BLOCKS + block] = sum over this block's share of i of
// vec(q)[i] * w[i] for q = q0 .. q0 + K - 1, vec(q) = V + q * ldv for
// q < nv and w itself for q == nv (so ||w||^2 comes out of the same pass).
// K is a compile-time count: FP64 FMAs are scarce on this part, a
// predicated-off FMA still takes its issue slot on the FP64 pipe, and small K
// keeps registers (and so occupancy) low. Every q's sum runs in the same
// order whatever K is, so results do not depend on how the vectors are
// grouped into launches.
template <int K>
__device__ __forceinline__ void multidot_body(const double* __restrict__ V, size_t ldv, int nv, int q0,
                                              const double* __restrict__ w, size_t N,
                                              double* __restrict__ partial) {
  __shared__ double sm[K][RED_THREADS / 32];
  const double* vp[K];
#pragma unroll
  for (int q = 0; q < K; ++q) vp[q] = q0 + q < nv ? V + (size_t)(q0 + q) * ldv : w;
  double acc[K];
#pragma unroll
  for (int q = 0; q < K; ++q) acc[q] = 0.0;
  const size_t stride = (size_t)RED_BLOCKS * RED_THREADS;
  for (size_t i = blockIdx.x * (size_t)RED_THREADS + threadIdx.x; i < N; i += stride) {
    const double wi = __ldg(w + i);
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q] = fma(__ldg(vp[q] + i), wi, acc[q]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double v = acc[q];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    if (lane == 0) sm[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double v = 0.0;
    for (int wv = 0; wv < RED_THREADS / 32; ++wv) v += sm[threadIdx.x][wv];
    partial[(size_t)(q0 + threadIdx.x) * RED_BLOCKS + blockIdx.x] = v;
  }
}

template <int K>
__global__ void __launch_bounds__(RED_THREADS) k_multidot(const double* __restrict__ V, size_t ldv, int q_base,
                                                          const double* __restrict__ w, size_t N,
                                                          double* __restrict__ partial) {
  dep_enter();
  multidot_body<K>(V, ldv, 1 << 30, q_base + blockIdx.y * K, w, N, partial);
}

// The same products for the device-resident FGMRES step: the vectors are
// V_0 .. V_j (j read from the step state) and, with with_w, w itself; block
// row y takes vectors 8y .. 8y + 7 of them (fewer in the last row, none past
// the end), dispatched to the compile-time count.
__global__ void __launch_bounds__(RED_THREADS) k_multidot_ks(const double* __restrict__ V, size_t ldv,
                                                             const KrylovState* __restrict__ ks, int with_w,
                                                             const double* __restrict__ w, size_t N,
                                                             double* __restrict__ partial) {
  dep_enter();
  const int nv = ks->j + 1, k = nv + with_w;
  const int q0 = blockIdx.y * MD_CHUNK, cnt = min(MD_CHUNK, k - q0);
  switch (cnt) {
    case 8: multidot_body<8>(V, ldv, nv, q0, w, N, partial); break;
    case 7: multidot_body<7>(V, ldv, nv, q0, w, N, partial); break;
    case 6: multidot_body<6>(V, ldv, nv, q0, w, N, partial); break;
    case 5: multidot_body<5>(V, ldv, nv, q0, w, N, partial); break;
    case 4: multidot_body<4>(V, ldv, nv, q0, w, N, partial); break;
    case 3: multidot_body<3>(V, ldv, nv, q0, w, N, partial); break;
    case 2: multidot_body<2>(V, ldv, nv, q0, w, N, partial); break;
    case 1: multidot_body<1>(V, ldv, nv, q0, w, N, partial); break;
    default: break;
  }
}

// out[q] = sum of the RED_BLOCKS partials of vector q (fixed tree); with ks,
// vectors q >= j + 1 + extra are absent (their blocks return).
__global__ void __launch_bounds__(RED_THREADS) k_reduce_partials(const double* __restrict__ partial,
                                                                 double* __restrict__ out,
                                                                 const KrylovState* __restrict__ ks, int extra) {
  dep_enter();
  __shared__ double sm[RED_THREADS / 32];
  const int q = blockIdx.x;
  if (ks && q >= ks->j + 1 + extra) return;
  double v = 0.0;
  for (int b = threadIdx.x; b < RED_BLOCKS; b += RED_THREADS) v += partial[(size_t)q * RED_BLOCKS + b];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int wv = 0; wv < RED_THREADS / 32; ++wv) t += sm[wv];
    out[q] = t;
  }
}

// *flag = 1.0 if some x[i] != 0 (flag cleared to 0.0 beforehand).
__global__ void k_any_nonzero(const double* __restrict__ x, size_t N, double* __restrict__ flag) {
  dep_enter();
  bool nz = false;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    nz |= x[i] != 0.0;
  if (__syncthreads_or(nz) && threadIdx.x == 0) *flag = 1.0;
}

// w[i] -= sum_q h[q] V[q][i]
__global__ void k_gs_update(const double* __restrict__ V, size_t ldv, int k, const double* __restrict__ h,
                            double* __restrict__ w, size_t N) {
  dep_enter();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    double t = w[i];
    for (int q = 0; q < k; ++q) t = fma(-__ldg(h + q), __ldg(V + (size_t)q * ldv + i), t);
    w[i] = t;
  }
}

// The same update (k = j + 1 from the step state when ks is given) on the
// reduction grid of k_multidot, and, when partial is given, the partial sums
// of the updated w's squares with k_multidot<1>'s order and tree: the norm of
// CGS2's second pass without another read of w.
__global__ void __launch_bounds__(RED_THREADS) k_gs_update_norm(const double* __restrict__ V, size_t ldv, int k_host,
                                                                const KrylovState* __restrict__ ks,
                                                                const double* __restrict__ h, double* __restrict__ w,
                                                                size_t N, double* __restrict__ partial) {
  dep_enter();
  const int k = ks ? ks->j + 1 : k_host;
  double acc = 0.0;
  const size_t stride = (size_t)RED_BLOCKS * RED_THREADS;
  for (size_t i = blockIdx.x * (size_t)RED_THREADS + threadIdx.x; i < N; i += stride) {
    double t = w[i];
    for (int q = 0; q < k; ++q) t = fma(-__ldg(h + q), __ldg(V + (size_t)q * ldv + i), t);
    w[i] = t;
    acc = fma(t, t, acc);
  }
  if (!partial) return;
  __shared__ double sm[RED_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
  if (lane == 0) sm[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int wv = 0; wv < RED_THREADS / 32; ++wv) v += sm[wv];
    partial[blockIdx.x] = v;
  }
}

struct Coefs {
  double c[72];
};

// x[i] += sum_q y[q] Z[q][i]
template <class TZ>
__global__ void k_add_combination(const TZ* __restrict__ Z, size_t ldz, int k, Coefs y, double* __restrict__ x,
                                  size_t N) {
  dep_enter();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    double t = x[i];
    for (int q = 0; q < k; ++q) t = fma(y.c[q], (double)Z[(size_t)q * ldz + i], t);
    x[i] = t;
  }
}

// y = a x + b y (one element; shared with the device-resident BiCGStab)
__device__ __forceinline__ double axpby_elem(double a, double x, double b, double y) { return a * x + b * y; }

__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, size_t N) {
  dep_enter();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    y[i] = axpby_elem(a, x[i], b, y[i]);
}

// y = a x
__global__ void k_scale(double a, const double* x, double* y, size_t N) {
  dep_enter();  // may run in place
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

// p = r + beta (p - omega v)
__device__ __forceinline__ double bicg_p_elem(double beta, double omega, double r, double v, double p) {
  return r + beta * (p - omega * v);
}

__global__ void k_bicg_p(double beta, double omega, const double* __restrict__ r, const double* __restrict__ v,
                         double* __restrict__ p, size_t N) {
  dep_enter();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    p[i] = bicg_p_elem(beta, omega, r[i], v[i], p[i]);
}

// ---- device-resident FGMRES cycle (state in KrylovState) -------------------
// The scalar recurrences below repeat the host loop's operations one by one
// with explicitly rounded FP64 operations (no fused multiply-add), as the
// host compiler evaluates them, so both paths give the same bits.
__global__ void k_ks_init(KrylovState* ks, double beta, double bnorm, int iters, int m, int maxiter, double tol) {
  dep_enter();
  const int t = threadIdx.x;
  for (int i = t; i <= m; i += blockDim.x) ks->g[i] = i == 0 ? beta : 0.0;
  if (t == 0) {
    ks->j = 0;
    ks->iters = iters;
    ks->stop = KS_RUN;
    ks->jend = 0;
    ks->m = m;
    ks->maxiter = maxiter;
    ks->tol = tol;
    ks->bnorm = bnorm;
    ks->rhn = 0.0;
  }
}

// out = V_j (FP32 rounded to nearest, or FP64 copy)
template <class TO>
__global__ void k_ks_take_vj(const double* __restrict__ V, size_t ldv, const KrylovState* __restrict__ ks,
                             TO* __restrict__ out, size_t N) {
  dep_enter();
  const double* v = V + (size_t)ks->j * ldv;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (TO)v[i];
}

// Z_j = z; widen = z in FP64 when given (the outer SpMV's input)
template <class TZ>
__global__ void k_ks_store_z(const TZ* __restrict__ z, TZ* __restrict__ Z, const KrylovState* __restrict__ ks,
                             double* __restrict__ widen, size_t N) {
  dep_enter();
  TZ* zj = Z + (size_t)ks->j * N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const TZ v = z[i];
    zj[i] = v;
    if (widen) widen[i] = (double)v;
  }
}

// Step j's column of the Hessenberg matrix from the two Gram-Schmidt passes,
// the previous rotations applied to it, a new rotation that zeroes its
// subdiagonal entry, and the stop decision: non-finite values (breakdown),
// h_{j+1,j} <= 1e-14 ||A z_j|| (happy breakdown: no v_{j+1}), the rotated
// residual |g_{j+1}| <= tol ||b|| or the iteration limit, the end of the
// cycle. Sets the loop condition of the graph's WHILE node.
__device__ int givens_step(KrylovState* __restrict__ ks, const double* __restrict__ scal, int slot_a, int slot_b,
                           int slot_n) {
  const int j = ks->j, m = ks->m;
  double* H = ks->H;
  const double wn0 = __dsqrt_rn(scal[slot_a + j + 1]);
  const double hn = __dsqrt_rn(scal[slot_n]);
  for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = __dadd_rn(scal[slot_a + i], scal[slot_b + i]);
  H[(size_t)(j + 1) * m + j] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
    H[(size_t)i * m + j] = __dadd_rn(__dmul_rn(ks->cs[i], a), __dmul_rn(ks->sn[i], c));
    H[(size_t)(i + 1) * m + j] = __dadd_rn(__dmul_rn(-ks->sn[i], a), __dmul_rn(ks->cs[i], c));
  }
  const double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
  double cj, sj;
  if (c == 0.0) {
    cj = 1.0;
    sj = 0.0;
  } else {
    const double d = __dsqrt_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(c, c)));
    cj = __ddiv_rn(a, d);
    sj = __ddiv_rn(c, d);
  }
  ks->cs[j] = cj;
  ks->sn[j] = sj;
  H[(size_t)j * m + j] = __dadd_rn(__dmul_rn(cj, a), __dmul_rn(sj, c));
  H[(size_t)(j + 1) * m + j] = 0.0;
  const double gj = ks->g[j];
  const double g1 = __dmul_rn(-sj, gj);
  ks->g[j + 1] = g1;
  ks->g[j] = __dmul_rn(cj, gj);
  const int iters = ks->iters + 1;
  ks->iters = iters;
  ks->jend = j + 1;
  int stop = KS_RUN;
  if (!isfinite(hn) || !isfinite(g1)) {
    stop = KS_BREAKDOWN;
  } else if (!(hn > __dmul_rn(1e-14, wn0))) {
    stop = KS_HAPPY;
  } else {
    ks->rhn = __ddiv_rn(1.0, hn);
    if (fabs(g1) <= __dmul_rn(ks->tol, ks->bnorm)) stop = KS_CONVERGED;
    else if (iters >= ks->maxiter) stop = KS_MAXITER;
    else if (j + 1 >= m) stop = KS_CYCLE_END;
  }
  ks->stop = stop;
  ks->j = j + 1;
  return stop;
}

__global__ void k_ks_givens(KrylovState* __restrict__ ks, const double* __restrict__ scal, int slot_a, int slot_b,
                            int slot_n, cudaGraphConditionalHandle cond, int use_cond) {
  dep_enter();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int stop = givens_step(ks, scal, slot_a, slot_b, slot_n);
  if (use_cond) cudaGraphSetConditional(cond, stop == KS_RUN ? 1u : 0u);
}

// V_{j+1} = w / h_{j+1,j} unless the step broke down (j already advanced)
__global__ void k_ks_scale_next(const KrylovState* __restrict__ ks, const double* __restrict__ w,
                                double* __restrict__ V, size_t ldv, size_t N) {
  dep_enter();
  const int stop = ks->stop;
  if (stop == KS_HAPPY || stop == KS_BREAKDOWN) return;
  const double a = ks->rhn;
  double* v = V + (size_t)ks->j * ldv;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    v[i] = a * w[i];
}

// y = R^{-1} g over the cycle's jend steps (back substitution)
__global__ void k_ks_backsolve(KrylovState* __restrict__ ks) {
  dep_enter();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (ks->stop == KS_BREAKDOWN) return;
  const int jend = ks->jend, m = ks->m;
  const double* H = ks->H;
  for (int i = jend - 1; i >= 0; --i) {
    double t = ks->g[i];
    for (int k = i + 1; k < jend; ++k) t = __dsub_rn(t, __dmul_rn(H[(size_t)i * m + k], ks->y[k]));
    ks->y[i] = __ddiv_rn(t, H[(size_t)i * m + i]);
  }
}

// x += sum_{q < jend} y_q Z_q (nothing after a breakdown)
template <class TZ>
__global__ void k_ks_combine(const TZ* __restrict__ Z, size_t ldz, const KrylovState* __restrict__ ks,
                             double* __restrict__ x, size_t N) {
  dep_enter();
  const int k = ks->stop == KS_BREAKDOWN ? 0 : ks->jend;
  const double* y = ks->y;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    double t = x[i];
    for (int q = 0; q < k; ++q) t = fma(y[q], (double)Z[(size_t)q * ldz + i], t);
    x[i] = t;
  }
}

__global__ void k_ks_export(const KrylovState* __restrict__ ks, double* __restrict__ scal) {
  dep_enter();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  scal[0] = (double)ks->iters;
  scal[1] = (double)ks->jend;
  scal[2] = (double)ks->stop;
}

// ---- batched steps: blockIdx.z selects the case ------------------------------
// Each case's arithmetic is the single-system kernels' (the same device
// functions, grids of the same shape per case), so a batched solve gives
// every case the bits it gets alone. A case takes part in a step when its
// restart cycle was running at the step's start (live, set by
// kb_step_begin); the finishing kernels serve the cases of the current
// restart round.
__global__ void kb_step_begin_k(const BCase* __restrict__ cases, int count) {
  dep_enter();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < count) *cases[c].live = cases[c].ks->stop == KS_RUN;
}

__global__ void kb_take_vj_k(const BCase* __restrict__ cases) {
  dep_enter();
  const BCase& c = cases[blockIdx.z];
  if (!*c.live) return;
  const double* v = c.V + (size_t)c.ks->j * c.N;
  float* out = c.lv[0].vb;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < c.N; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)v[i];
}

__global__ void kb_store_z_k(const BCase* __restrict__ cases) {
  dep_enter();
  const BCase& c = cases[blockIdx.z];
  if (!*c.live) return;
  const float* z = c.lv[0].vx;
  float* zj = c.Z + (size_t)c.ks->j * c.N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < c.N; i += (size_t)gridDim.x * blockDim.x) {
    const float v = z[i];
    zj[i] = v;
    c.kt[i] = (double)v;
  }
}

__global__ void __launch_bounds__(RED_THREADS) kb_multidot_k(const BCase* __restrict__ cases, int with_w) {
  dep_enter();
  const BCase& c = cases[blockIdx.z];
  if (!*c.live) return;
  const int nv = c.ks->j + 1, k = nv + with_w;
  const int q0 = blockIdx.y * MD_CHUNK, cnt = min(MD_CHUNK, k - q0);
  switch (cnt) {
    case 8: multidot_body<8>(c.V, c.N, nv, q0, c.w, c.N, c.red); break;
    case 7: multidot_body<7>(c.V, c.N, nv, q0, c.w, c.N, c.red); break;
    case 6: multidot_body<6>(c.V, c.N, nv, q0, c.w, c.N, c.red); break;
    case 5: multidot_body<5>(c.V, c.N, nv, q0, c.w, c.N, c.red); break;
    case 4: multidot_body<4>(c.V, c.N, nv, q0, c.w, c.N, c.red); break;
    case 3: multidot_body<3>(c.V, c.N, nv, q0, c.w, c.N, c.red); break;
    case 2: multidot_body<2>(c.V, c.N, nv, q0, c.w, c.N, c.red); break;
    case 1: multidot_body<1>(c.V, c.N, nv, q0, c.w, c.N, c.red); break;
    default: break;
  }
}

// the partials of vectors q < nq (nq: j + 1 + extra when per_step, else 1)
// to scal[slot + q]; the case takes part when live (per_step) or in the round
__global__ void __launch_bounds__(RED_THREADS) kb_reduce_k(const BCase* __restrict__ cases, int slot, int extra,
                                                          int per_step) {
  dep_enter();
  const BCase& c = cases[blockIdx.z];
  if (per_step ? !*c.live : !*c.round) return;
  const int q = blockIdx.x;
  if (q >= (per_step ? c.ks->j + 1 + extra : 1)) return;
  __shared__ double sm[RED_THREADS / 32];
  double v = 0.0;
  for (int b = threadIdx.x; b < RED_BLOCKS; b += RED_THREADS) v += c.red[(size_t)q * RED_BLOCKS + b];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int wv = 0; wv < RED_THREADS / 32; ++wv) t += sm[wv];
    c.scal[slot + q] = t;
  }
}

__global__ void __launch_bounds__(RED_THREADS) kb_gs_update_k(const BCase* __restrict__ cases, int hslot, int norm) {
  dep_enter();
  const BCase& c = cases[blockIdx.z];
  if (!*c.live) return;
  const int k = c.ks->j + 1;
  const double* h = c.scal + hslot;
  double acc = 0.0;
  const size_t stride = (size_t)RED_BLOCKS * RED_THREADS;
  for (size_t i = blockIdx.x * (size_t)RED_THREADS + threadIdx.x; i < c.N; i += stride) {
    double t = c.w[i];
    for (int q = 0; q < k; ++q) t = fma(-__ldg(h + q), __ldg(c.V + (size_t)q * c.N + i), t);
    c.w[i] = t;
    acc = fma(t, t, acc);
  }
  if (!norm) return;
  __shared__ double sm[RED_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
  if (lane == 0) sm[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int wv = 0; wv < RED_THREADS / 32; ++wv) v += sm[wv];
    c.red[blockIdx.x] = v;
  }
}

// Givens update and stop test of every live case; the loop continues while
// one of them still runs.
__global__ void kb_givens_k(const BCase* __restrict__ cases, int count, cudaGraphConditionalHandle cond) {
  dep_enter();
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < count; c += blockDim.x) {
    const BCase& bc = cases[c];
    if (!*bc.live) continue;
    if (givens_step(bc.ks, bc.scal, SLOT_A, SLOT_B, SLOT_N) == KS_RUN) atomicOr(&any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) cudaGraphSetConditional(cond, any ? 1u : 0u);
}

__global__ void kb_scale_next_k(const BCase* __restrict__ cases) {
  dep_enter();
  const BCase& c = cases[blockIdx.z];
  if (!*c.live) return;
  const int stop = c.ks->stop;
  if (stop == KS_HAPPY || stop == KS_BREAKDOWN) return;
  const double a = c.ks->rhn;
  double* v = c.V + (size_t)c.ks->j * c.N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < c.N; i += (size_t)gridDim.x * blockDim.x)
    v[i] = a * c.w[i];
}

// back substitution (one thread per case), then x += Z y
__global__ void kb_backsolve_k(const BCase* __restrict__ cases, int count) {
  dep_enter();
  const int ci = blockIdx.x * blockDim.x + threadIdx.x;
  if (ci >= count || !*cases[ci].round) return;
  KrylovState* ks = cases[ci].ks;
  if (ks->stop == KS_BREAKDOWN) return;
  const int jend = ks->jend, m = ks->m;
  const double* H = ks->H;
  for (int i = jend - 1; i >= 0; --i) {
    double t = ks->g[i];
    for (int k = i + 1; k < jend; ++k) t = __dsub_rn(t, __dmul_rn(H[(size_t)i * m + k], ks->y[k]));
    ks->y[i] = __ddiv_rn(t, H[(size_t)i * m + i]);
  }
}

__global__ void kb_combine_k(const BCase* __restrict__ cases) {
  dep_enter();
  const BCase& c = cases[blockIdx.z];
  if (!*c.round) return;
  const int k = c.ks->stop == KS_BREAKDOWN ? 0 : c.ks->jend;
  const double* y = c.ks->y;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < c.N; i += (size_t)gridDim.x * blockDim.x) {
    double t = c.x[i];
    for (int q = 0; q < k; ++q) t = fma(y[q], (double)c.Z[(size_t)q * c.N + i], t);
    c.x[i] = t;
  }
}

// partials of ||r||^2 (k_multidot<1>'s order and tree) and the cycle outcome
__global__ void __launch_bounds__(RED_THREADS) kb_norm_r_k(const BCase* __restrict__ cases) {
  dep_enter();
  const BCase& c = cases[blockIdx.z];
  if (!*c.round) return;
  multidot_body<1>(c.r, c.N, 1 << 30, 0, c.r, c.N, c.red);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c.scal[SLOT_S] = (double)c.ks->iters;
    c.scal[SLOT_S + 1] = (double)c.ks->jend;
    c.scal[SLOT_S + 2] = (double)c.ks->stop;
  }
}

// every case's ||r||^2 and cycle outcome into one array (one read for all)
__global__ void kb_gather_out_k(const BCase* __restrict__ cases, int count, double* __restrict__ out) {
  dep_enter();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= count) return;
  const double* sc = cases[c].scal;
  out[4 * c] = sc[SLOT_N];
  out[4 * c + 1] = sc[SLOT_S];
  out[4 * c + 2] = sc[SLOT_S + 1];
  out[4 * c + 3] = sc[SLOT_S + 2];
}

// ---- device-resident BiCGStab (state in BicgState, scalars in scal) ----------
// The scalars are formed with explicitly rounded operations in the order the
// host-driven loop evaluates them, and the vector updates use the same
// element functions, so both loops give the same bits.
__global__ void k_bs_init(BicgState* bs, int it, int maxiter, double tol, double bnorm, int first) {
  dep_enter();
  if (threadIdx.x != 0) return;
  bs->it = it;
  bs->stop = BS_RUN;
  bs->first = first;
  bs->maxiter = maxiter;
  bs->tol = tol;
  bs->bnorm = bnorm;
  if (first == 2) {  // a fresh solve: the host loop's starting values
    bs->rho_old = 1.0;
    bs->alpha = 1.0;
    bs->omega = 1.0;
    bs->first = 1;
  }
}

__global__ void k_bs_rho(BicgState* __restrict__ bs, const double* __restrict__ scal) {
  dep_enter();
  if (threadIdx.x != 0 || bs->stop != BS_RUN) return;
  const double rho = scal[SLOT_A];
  bs->rho = rho;
  if (rho == 0.0 || !isfinite(rho)) {
    bs->stop = BS_BREAK;
    return;
  }
  if (!bs->first) bs->beta = __dmul_rn(__ddiv_rn(rho, bs->rho_old), __ddiv_rn(bs->alpha, bs->omega));
}

__global__ void k_bs_p(const BicgState* __restrict__ bs, const double* __restrict__ r, const double* __restrict__ v,
                       double* __restrict__ p, size_t N) {
  dep_enter();
  if (bs->stop != BS_RUN) return;
  const bool first = bs->first;
  const double beta = bs->beta, omega = bs->omega;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    p[i] = first ? r[i] : bicg_p_elem(beta, omega, r[i], v[i], p[i]);
}

__global__ void k_bs_alpha(BicgState* __restrict__ bs, const double* __restrict__ scal) {
  dep_enter();
  if (threadIdx.x != 0 || bs->stop != BS_RUN) return;
  bs->first = 0;
  const double den = scal[SLOT_A];
  if (den == 0.0 || !isfinite(den)) {
    bs->stop = BS_BREAK;
    return;
  }
  bs->alpha = __ddiv_rn(bs->rho, den);
}

// s = r - alpha v (the host loop: s = r, then s = (-alpha) v + 1 s)
__global__ void k_bs_s(const BicgState* __restrict__ bs, const double* __restrict__ r, const double* __restrict__ v,
                       double* __restrict__ sv, size_t N) {
  dep_enter();
  if (bs->stop != BS_RUN) return;
  const double a = -bs->alpha;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    sv[i] = axpby_elem(a, v[i], 1.0, r[i]);
}

__global__ void k_bs_snorm(BicgState* __restrict__ bs, const double* __restrict__ scal) {
  dep_enter();
  if (threadIdx.x != 0 || bs->stop != BS_RUN) return;
  bs->it = bs->it + 1;
  const double snrm = __dsqrt_rn(scal[SLOT_N]);
  if (snrm <= __dmul_rn(bs->tol, bs->bnorm)) bs->stop = BS_S_SMALL;
}

__global__ void k_bs_omega(BicgState* __restrict__ bs, const double* __restrict__ scal) {
  dep_enter();
  if (threadIdx.x != 0 || bs->stop != BS_RUN) return;
  const double ts = scal[SLOT_A], tt = scal[SLOT_A + 1];
  if (tt == 0.0 || !isfinite(tt)) {
    bs->stop = BS_BREAK;
    return;
  }
  bs->omega = __ddiv_rn(ts, tt);
}

// x += alpha ph + omega sh (ph and sh consecutive, cycle precision)
template <class TZ>
__global__ void k_bs_x(const BicgState* __restrict__ bs, const TZ* __restrict__ ph, double* __restrict__ x, size_t N) {
  dep_enter();
  if (bs->stop != BS_RUN) return;
  const double a = bs->alpha, o = bs->omega;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    double t = x[i];
    t = fma(a, (double)ph[i], t);
    t = fma(o, (double)ph[N + i], t);
    x[i] = t;
  }
}

// r = s - omega t (the host loop: r = s, then r = (-omega) t + 1 r)
__global__ void k_bs_r(const BicgState* __restrict__ bs, const double* __restrict__ sv, const double* __restrict__ t,
                       double* __restrict__ r, size_t N) {
  dep_enter();
  if (bs->stop != BS_RUN) return;
  const double a = -bs->omega;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    r[i] = axpby_elem(a, t[i], 1.0, sv[i]);
}

// end of an iteration: rho_old, the residual test, omega = 0, the limit;
// the loop runs on while nothing happened
__global__ void k_bs_export(const BicgState* __restrict__ bs, double* __restrict__ scal) {
  dep_enter();
  if (threadIdx.x != 0) return;
  scal[SLOT_S] = (double)bs->it;
  scal[SLOT_S + 1] = (double)bs->stop;
  scal[SLOT_S + 2] = bs->alpha;
}

__global__ void k_bs_end(BicgState* __restrict__ bs, const double* __restrict__ scal,
                         cudaGraphConditionalHandle cond) {
  dep_enter();
  if (threadIdx.x != 0) return;
  if (bs->stop == BS_RUN) {
    bs->rho_old = bs->rho;
    const double rn = __dsqrt_rn(scal[SLOT_N]);
    if (rn <= __dmul_rn(bs->tol, bs->bnorm)) bs->stop = BS_R_SMALL;
    else if (bs->omega == 0.0) bs->stop = BS_OMEGA0;
    else if (bs->it >= bs->maxiter) bs->stop = BS_MAXITER;
  }
  cudaGraphSetConditional(cond, bs->stop == BS_RUN ? 1u : 0u);
}

unsigned vgrid(size_t N) {
  unsigned g = grid_for(N, 256);
  return g > 148u * 16u ? 148u * 16u : g;
}

}  // namespace

bcs_status multidot(Solver* s, const double* V, size_t ldv, int k, const double* w, size_t N, int slot) {
  if (k <= 0) return BCS_OK;
  BCS_ALLOC(s, s->red, (size_t)72 * RED_BLOCKS);
  if (k > 72) return s->fail(BCS_EINVAL, "too many vectors in one multidot");
  const int full = k / MD_CHUNK, rem = k % MD_CHUNK;
  if (full > 0)
    BCS_LAUNCH_DEP(s, K_BLAS, 8.0 * N * (full * MD_CHUNK + full), 2.0 * N * full * MD_CHUNK, k_multidot<MD_CHUNK>,
               dim3(RED_BLOCKS, full), RED_THREADS, 0, V, ldv, 0, w, N, s->red.p);
  const int qb = full * MD_CHUNK;
  switch (rem) {
#define BCS_MD_TAIL(R)                                                                                   \
  case R:                                                                                                \
    BCS_LAUNCH_DEP(s, K_BLAS, 8.0 * N * (R + 1), 2.0 * N * R, k_multidot<R>, dim3(RED_BLOCKS, 1), RED_THREADS, 0, \
               V, ldv, qb, w, N, s->red.p);                                                              \
    break;
    BCS_MD_TAIL(1) BCS_MD_TAIL(2) BCS_MD_TAIL(3) BCS_MD_TAIL(4) BCS_MD_TAIL(5) BCS_MD_TAIL(6) BCS_MD_TAIL(7)
#undef BCS_MD_TAIL
    default: break;
  }
  BCS_LAUNCH_DEP(s, K_BLAS, 8.0 * k * RED_BLOCKS, 0, k_reduce_partials, k, RED_THREADS, 0, s->red.p, s->scal.p + slot,
             (const KrylovState*)nullptr, 0);
  return BCS_OK;
}

bcs_status dot(Solver* s, const double* x, const double* y, size_t N, int slot) {
  return multidot(s, x, N, 1, y, N, slot);
}

bcs_status any_nonzero(Solver* s, const double* x, size_t N, int slot) {
  BCS_CU(s, cudaMemsetAsync(s->scal.p + slot, 0, sizeof(double), s->stream));
  BCS_LAUNCH_DEP(s, K_BLAS, 8.0 * N, 0, k_any_nonzero, RED_BLOCKS, RED_THREADS, 0, x, N, s->scal.p + slot);
  return BCS_OK;
}

bcs_status fetch_scalars(Solver* s, int count) {
  BCS_CU(s, cudaMemcpyAsync(s->hscal, s->scal.p, count * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  ++s->host_syncs;
  return BCS_OK;
}

bcs_status gs_update(Solver* s, const double* V, size_t ldv, int k, const double* hdev, double* w, size_t N) {
  BCS_LAUNCH_DEP(s, K_BLAS, 8.0 * N * (k + 2), 2.0 * N * k, k_gs_update, vgrid(N), 256, 0, V, ldv, k, hdev, w, N);
  return BCS_OK;
}

bcs_status gs_update_norm(Solver* s, const double* V, size_t ldv, int k, const double* hdev, double* w, size_t N,
                          int slot) {
  BCS_ALLOC(s, s->red, (size_t)72 * RED_BLOCKS);
  BCS_LAUNCH_DEP(s, K_BLAS, 8.0 * N * (k + 2), 2.0 * N * (k + 1), k_gs_update_norm, RED_BLOCKS, RED_THREADS, 0, V, ldv, k,
             (const KrylovState*)nullptr, hdev, w, N, s->red.p);
  BCS_LAUNCH_DEP(s, K_BLAS, 8.0 * RED_BLOCKS, 0, k_reduce_partials, 1, RED_THREADS, 0, s->red.p, s->scal.p + slot,
             (const KrylovState*)nullptr, 0);
  return BCS_OK;
}

bcs_status ks_init(Solver* s, KrylovState* ks, double beta, double bnorm, int iters, int m, int maxiter, double tol) {
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, k_ks_init, 1, 128, 0, ks, beta, bnorm, iters, m, maxiter, tol);
  return BCS_OK;
}

bcs_status ks_take_vj(Solver* s, const double* V, size_t ldv, const KrylovState* ks, void* out, bool to_float,
                      size_t N) {
  if (to_float)
    BCS_LAUNCH_DEP(s, K_CAST, 12.0 * N, 0, k_ks_take_vj<float>, vgrid(N), 256, 0, V, ldv, ks, (float*)out, N);
  else
    BCS_LAUNCH_DEP(s, K_BLAS, 16.0 * N, 0, k_ks_take_vj<double>, vgrid(N), 256, 0, V, ldv, ks, (double*)out, N);
  return BCS_OK;
}

bcs_status ks_store_z(Solver* s, const void* zsrc, bool z_float, void* Z, const KrylovState* ks, double* widen,
                      size_t N) {
  if (z_float)
    BCS_LAUNCH_DEP(s, K_CAST, (12.0 + (widen ? 8.0 : 0.0)) * N, 0, k_ks_store_z<float>, vgrid(N), 256, 0,
               (const float*)zsrc, (float*)Z, ks, widen, N);
  else
    BCS_LAUNCH_DEP(s, K_BLAS, (16.0 + (widen ? 8.0 : 0.0)) * N, 0, k_ks_store_z<double>, vgrid(N), 256, 0,
               (const double*)zsrc, (double*)Z, ks, widen, N);
  return BCS_OK;
}

// bytes and flops are counted for the largest step (j = m - 1); the graph's
// launch statistics use these per step
bcs_status ks_multidot(Solver* s, const double* V, size_t ldv, const KrylovState* ks, const double* w, bool with_w,
                       size_t N, int slot) {
  const int kmax = s->cfg.restart + (with_w ? 1 : 0);
  if (kmax > 72) return s->fail(BCS_EINVAL, "too many vectors in one multidot");
  BCS_ALLOC(s, s->red, (size_t)72 * RED_BLOCKS);
  const unsigned chunks = (unsigned)((kmax + MD_CHUNK - 1) / MD_CHUNK);
  BCS_LAUNCH_DEP(s, K_BLAS, 8.0 * N * (kmax + 1), 2.0 * N * kmax, k_multidot_ks, dim3(RED_BLOCKS, chunks), RED_THREADS, 0,
             V, ldv, ks, with_w ? 1 : 0, w, N, s->red.p);
  BCS_LAUNCH_DEP(s, K_BLAS, 8.0 * kmax * RED_BLOCKS, 0, k_reduce_partials, kmax, RED_THREADS, 0, s->red.p,
             s->scal.p + slot, ks, with_w ? 1 : 0);
  return BCS_OK;
}

bcs_status ks_gs_update(Solver* s, const double* V, size_t ldv, const KrylovState* ks, const double* hdev, double* w,
                        size_t N, int norm_slot) {
  const int kmax = s->cfg.restart;
  BCS_ALLOC(s, s->red, (size_t)72 * RED_BLOCKS);
  BCS_LAUNCH_DEP(s, K_BLAS, 8.0 * N * (kmax + 2), 2.0 * N * kmax, k_gs_update_norm, RED_BLOCKS, RED_THREADS, 0, V, ldv, 0,
             ks, hdev, w, N, norm_slot >= 0 ? s->red.p : nullptr);
  if (norm_slot >= 0)
    BCS_LAUNCH_DEP(s, K_BLAS, 8.0 * RED_BLOCKS, 0, k_reduce_partials, 1, RED_THREADS, 0, s->red.p,
               s->scal.p + norm_slot, (const KrylovState*)nullptr, 0);
  return BCS_OK;
}

bcs_status ks_givens(Solver* s, KrylovState* ks, int slot_a, int slot_b, int slot_n, cudaGraphConditionalHandle cond) {
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, k_ks_givens, 1, 32, 0, ks, (const double*)s->scal.p, slot_a, slot_b, slot_n, cond, 1);
  return BCS_OK;
}

bcs_status ks_scale_next(Solver* s, const KrylovState* ks, const double* w, double* V, size_t ldv, size_t N) {
  BCS_LAUNCH_DEP(s, K_BLAS, 16.0 * N, 1.0 * N, k_ks_scale_next, vgrid(N), 256, 0, ks, w, V, ldv, N);
  return BCS_OK;
}

bcs_status ks_finish_cycle(Solver* s, KrylovState* ks, const void* Z, bool z_float, double* x, size_t N) {
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, k_ks_backsolve, 1, 32, 0, ks);
  const double k = s->cfg.restart;
  if (z_float)
    BCS_LAUNCH_DEP(s, K_BLAS, (4.0 * k + 16.0) * N, 2.0 * N * k, k_ks_combine<float>, vgrid(N), 256, 0, (const float*)Z,
               N, (const KrylovState*)ks, x, N);
  else
    BCS_LAUNCH_DEP(s, K_BLAS, (8.0 * k + 16.0) * N, 2.0 * N * k, k_ks_combine<double>, vgrid(N), 256, 0,
               (const double*)Z, N, (const KrylovState*)ks, x, N);
  return BCS_OK;
}

bcs_status ks_export(Solver* s, const KrylovState* ks, int slot) {
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, k_ks_export, 1, 32, 0, ks, s->scal.p + slot);
  return BCS_OK;
}

bcs_status add_combination(Solver* s, const void* Z, bool z_float, size_t ldz, int k, const double* y, double* x,
                           size_t N) {
  if (k > 72) return s->fail(BCS_EINVAL, "too many vectors in one combination");
  Coefs c{};
  for (int q = 0; q < k; ++q) c.c[q] = y[q];
  if (z_float)
    BCS_LAUNCH_DEP(s, K_BLAS, (4.0 * k + 16.0) * N, 2.0 * N * k, k_add_combination<float>, vgrid(N), 256, 0,
               (const float*)Z, ldz, k, c, x, N);
  else
    BCS_LAUNCH_DEP(s, K_BLAS, (8.0 * k + 16.0) * N, 2.0 * N * k, k_add_combination<double>, vgrid(N), 256, 0,
               (const double*)Z, ldz, k, c, x, N);
  return BCS_OK;
}

bcs_status axpby(Solver* s, double a, const double* x, double b, double* y, size_t N) {
  BCS_LAUNCH_DEP(s, K_BLAS, 24.0 * N, 3.0 * N, k_axpby, vgrid(N), 256, 0, a, x, b, y, N);
  return BCS_OK;
}

bcs_status scale_copy(Solver* s, double a, const double* x, double* y, size_t N) {
  BCS_LAUNCH_DEP(s, K_BLAS, 16.0 * N, 1.0 * N, k_scale, vgrid(N), 256, 0, a, x, y, N);
  return BCS_OK;
}

bcs_status bicg_p_update(Solver* s, double beta, double omega, const double* r, const double* v, double* p,
                         size_t N) {
  BCS_LAUNCH_DEP(s, K_BLAS, 32.0 * N, 4.0 * N, k_bicg_p, vgrid(N), 256, 0, beta, omega, r, v, p, N);
  return BCS_OK;
}



// grid of the element-wise batched kernels: the largest case's
unsigned bgrid(size_t maxN) { return vgrid(maxN); }

bcs_status kb_step_begin(Solver* s, const BCase* cases, int count) {
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, kb_step_begin_k, grid_for(count, 64), 64, 0, cases, count);
  return BCS_OK;
}

bcs_status kb_take_vj(Solver* s, const BCase* cases, int count, size_t maxN) {
  BCS_LAUNCH_DEP(s, K_CAST, 12.0 * maxN * count, 0, kb_take_vj_k, dim3(bgrid(maxN), 1, count), 256, 0, cases);
  return BCS_OK;
}

bcs_status kb_store_z(Solver* s, const BCase* cases, int count, size_t maxN) {
  BCS_LAUNCH_DEP(s, K_CAST, 16.0 * maxN * count, 0, kb_store_z_k, dim3(bgrid(maxN), 1, count), 256, 0, cases);
  return BCS_OK;
}

bcs_status kb_multidot(Solver* s, const BCase* cases, int count, bool with_w, int kmax, int slot) {
  const unsigned chunks = (unsigned)((kmax + MD_CHUNK - 1) / MD_CHUNK);
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, kb_multidot_k, dim3(RED_BLOCKS, chunks, count), RED_THREADS, 0, cases, with_w ? 1 : 0);
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, kb_reduce_k, dim3(kmax, 1, count), RED_THREADS, 0, cases, slot, with_w ? 1 : 0, 1);
  return BCS_OK;
}

bcs_status kb_gs_update(Solver* s, const BCase* cases, int count, int hslot, int nslot) {
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, kb_gs_update_k, dim3(RED_BLOCKS, 1, count), RED_THREADS, 0, cases, hslot,
             nslot >= 0 ? 1 : 0);
  if (nslot >= 0) BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, kb_reduce_k, dim3(1, 1, count), RED_THREADS, 0, cases, nslot, 0, 1);
  return BCS_OK;
}

bcs_status kb_givens(Solver* s, const BCase* cases, int count, cudaGraphConditionalHandle cond) {
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, kb_givens_k, 1, 64, 0, cases, count, cond);
  return BCS_OK;
}

bcs_status kb_scale_next(Solver* s, const BCase* cases, int count, size_t maxN) {
  BCS_LAUNCH_DEP(s, K_BLAS, 16.0 * maxN * count, 0, kb_scale_next_k, dim3(bgrid(maxN), 1, count), 256, 0, cases);
  return BCS_OK;
}

bcs_status kb_finish(Solver* s, const BCase* cases, int count, size_t maxN) {
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, kb_backsolve_k, grid_for(count, 32), 32, 0, cases, count);
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, kb_combine_k, dim3(bgrid(maxN), 1, count), 256, 0, cases);
  return BCS_OK;
}

bcs_status kb_norm_r(Solver* s, const BCase* cases, int count) {
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, kb_norm_r_k, dim3(RED_BLOCKS, 1, count), RED_THREADS, 0, cases);
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, kb_reduce_k, dim3(1, 1, count), RED_THREADS, 0, cases, SLOT_N, 0, 0);
  return BCS_OK;
}

bcs_status kb_gather_out(Solver* s, const BCase* cases, int count, double* out) {
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, kb_gather_out_k, grid_for(count, 64), 64, 0, cases, count, out);
  return BCS_OK;
}

bcs_status bs_init(Solver* s, BicgState* bs, int it, int maxiter, double tol, double bnorm, int first) {
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, k_bs_init, 1, 32, 0, bs, it, maxiter, tol, bnorm, first);
  return BCS_OK;
}
bcs_status bs_rho(Solver* s, BicgState* bs) {
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, k_bs_rho, 1, 32, 0, bs, (const double*)s->scal.p);
  return BCS_OK;
}
bcs_status bs_p_update(Solver* s, const BicgState* bs, const double* r, const double* v, double* p, size_t N) {
  BCS_LAUNCH_DEP(s, K_BLAS, 32.0 * N, 4.0 * N, k_bs_p, vgrid(N), 256, 0, bs, r, v, p, N);
  return BCS_OK;
}
bcs_status bs_alpha(Solver* s, BicgState* bs) {
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, k_bs_alpha, 1, 32, 0, bs, (const double*)s->scal.p);
  return BCS_OK;
}
bcs_status bs_s_update(Solver* s, const BicgState* bs, const double* r, const double* v, double* sv, size_t N) {
  BCS_LAUNCH_DEP(s, K_BLAS, 24.0 * N, 3.0 * N, k_bs_s, vgrid(N), 256, 0, bs, r, v, sv, N);
  return BCS_OK;
}
bcs_status bs_snorm(Solver* s, BicgState* bs) {
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, k_bs_snorm, 1, 32, 0, bs, (const double*)s->scal.p);
  return BCS_OK;
}
bcs_status bs_omega(Solver* s, BicgState* bs) {
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, k_bs_omega, 1, 32, 0, bs, (const double*)s->scal.p);
  return BCS_OK;
}
bcs_status bs_x_update(Solver* s, const BicgState* bs, const void* ph, bool z_float, double* x, size_t N) {
  if (z_float)
    BCS_LAUNCH_DEP(s, K_BLAS, 24.0 * N, 4.0 * N, k_bs_x<float>, vgrid(N), 256, 0, bs, (const float*)ph, x, N);
  else
    BCS_LAUNCH_DEP(s, K_BLAS, 32.0 * N, 4.0 * N, k_bs_x<double>, vgrid(N), 256, 0, bs, (const double*)ph, x, N);
  return BCS_OK;
}
bcs_status bs_r_update(Solver* s, const BicgState* bs, const double* sv, const double* t, double* r, size_t N) {
  BCS_LAUNCH_DEP(s, K_BLAS, 24.0 * N, 3.0 * N, k_bs_r, vgrid(N), 256, 0, bs, sv, t, r, N);
  return BCS_OK;
}
bcs_status bs_end(Solver* s, BicgState* bs, cudaGraphConditionalHandle cond) {
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, k_bs_end, 1, 32, 0, bs, (const double*)s->scal.p, cond);
  return BCS_OK;
}

bcs_status bs_export(Solver* s, const BicgState* bs) {
  BCS_LAUNCH_DEP(s, K_BLAS, 0, 0, k_bs_export, 1, 32, 0, bs, s->scal.p);
  return BCS_OK;
}

}  // namespace bcs
