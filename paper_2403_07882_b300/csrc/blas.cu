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
// V[q][i] * w[i], for q = q_base + blockIdx.y * K + (0 .. K-1). K is a
// compile-time count: FP64 FMAs are scarce on this part, a predicated-off FMA
// still takes its issue slot on the FP64 pipe, and small K keeps registers
// (and so occupancy) low.
template <int K>
__global__ void __launch_bounds__(RED_THREADS) k_multidot(const double* __restrict__ V, size_t ldv, int q_base,
                                                          const double* __restrict__ w, size_t N,
                                                          double* __restrict__ partial) {
  __shared__ double sm[K][RED_THREADS / 32];
  const int q0 = q_base + blockIdx.y * K;
  double acc[K];
#pragma unroll
  for (int q = 0; q < K; ++q) acc[q] = 0.0;
  const size_t stride = (size_t)RED_BLOCKS * RED_THREADS;
  for (size_t i = blockIdx.x * (size_t)RED_THREADS + threadIdx.x; i < N; i += stride) {
    const double wi = __ldg(w + i);
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q] = fma(__ldg(V + (size_t)(q0 + q) * ldv + i), wi, acc[q]);
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

// out[q] = sum of the RED_BLOCKS partials of vector q (fixed tree).
__global__ void __launch_bounds__(RED_THREADS) k_reduce_partials(const double* __restrict__ partial,
                                                                 double* __restrict__ out) {
  __shared__ double sm[RED_THREADS / 32];
  const int q = blockIdx.x;
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
  bool nz = false;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    nz |= x[i] != 0.0;
  if (__syncthreads_or(nz) && threadIdx.x == 0) *flag = 1.0;
}

// w[i] -= sum_q h[q] V[q][i]
__global__ void k_gs_update(const double* __restrict__ V, size_t ldv, int k, const double* __restrict__ h,
                            double* __restrict__ w, size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    double t = w[i];
    for (int q = 0; q < k; ++q) t = fma(-__ldg(h + q), __ldg(V + (size_t)q * ldv + i), t);
    w[i] = t;
  }
}

struct Coefs {
  double c[72];
};

// x[i] += sum_q y[q] Z[q][i]
template <class TZ>
__global__ void k_add_combination(const TZ* __restrict__ Z, size_t ldz, int k, Coefs y, double* __restrict__ x,
                                  size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    double t = x[i];
    for (int q = 0; q < k; ++q) t = fma(y.c[q], (double)Z[(size_t)q * ldz + i], t);
    x[i] = t;
  }
}

// y = a x + b y
__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

// y = a x
__global__ void k_scale(double a, const double* x, double* y, size_t N) {  // may run in place
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

// p = r + beta (p - omega v)
__global__ void k_bicg_p(double beta, double omega, const double* __restrict__ r, const double* __restrict__ v,
                         double* __restrict__ p, size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    p[i] = r[i] + beta * (p[i] - omega * v[i]);
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
    BCS_LAUNCH(s, K_BLAS, 8.0 * N * (full * MD_CHUNK + full), 2.0 * N * full * MD_CHUNK, k_multidot<MD_CHUNK>,
               dim3(RED_BLOCKS, full), RED_THREADS, 0, V, ldv, 0, w, N, s->red.p);
  const int qb = full * MD_CHUNK;
  switch (rem) {
#define BCS_MD_TAIL(R)                                                                                   \
  case R:                                                                                                \
    BCS_LAUNCH(s, K_BLAS, 8.0 * N * (R + 1), 2.0 * N * R, k_multidot<R>, dim3(RED_BLOCKS, 1), RED_THREADS, 0, \
               V, ldv, qb, w, N, s->red.p);                                                              \
    break;
    BCS_MD_TAIL(1) BCS_MD_TAIL(2) BCS_MD_TAIL(3) BCS_MD_TAIL(4) BCS_MD_TAIL(5) BCS_MD_TAIL(6) BCS_MD_TAIL(7)
#undef BCS_MD_TAIL
    default: break;
  }
  BCS_LAUNCH(s, K_BLAS, 8.0 * k * RED_BLOCKS, 0, k_reduce_partials, k, RED_THREADS, 0, s->red.p, s->scal.p + slot);
  return BCS_OK;
}

bcs_status dot(Solver* s, const double* x, const double* y, size_t N, int slot) {
  return multidot(s, x, N, 1, y, N, slot);
}

bcs_status any_nonzero(Solver* s, const double* x, size_t N, int slot) {
  BCS_CU(s, cudaMemsetAsync(s->scal.p + slot, 0, sizeof(double), s->stream));
  BCS_LAUNCH(s, K_BLAS, 8.0 * N, 0, k_any_nonzero, RED_BLOCKS, RED_THREADS, 0, x, N, s->scal.p + slot);
  return BCS_OK;
}

bcs_status fetch_scalars(Solver* s, int count) {
  BCS_CU(s, cudaMemcpyAsync(s->hscal, s->scal.p, count * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  return BCS_OK;
}

bcs_status gs_update(Solver* s, const double* V, size_t ldv, int k, const double* hdev, double* w, size_t N) {
  BCS_LAUNCH(s, K_BLAS, 8.0 * N * (k + 2), 2.0 * N * k, k_gs_update, vgrid(N), 256, 0, V, ldv, k, hdev, w, N);
  return BCS_OK;
}

bcs_status add_combination(Solver* s, const void* Z, bool z_float, size_t ldz, int k, const double* y, double* x,
                           size_t N) {
  if (k > 72) return s->fail(BCS_EINVAL, "too many vectors in one combination");
  Coefs c{};
  for (int q = 0; q < k; ++q) c.c[q] = y[q];
  if (z_float)
    BCS_LAUNCH(s, K_BLAS, (4.0 * k + 16.0) * N, 2.0 * N * k, k_add_combination<float>, vgrid(N), 256, 0,
               (const float*)Z, ldz, k, c, x, N);
  else
    BCS_LAUNCH(s, K_BLAS, (8.0 * k + 16.0) * N, 2.0 * N * k, k_add_combination<double>, vgrid(N), 256, 0,
               (const double*)Z, ldz, k, c, x, N);
  return BCS_OK;
}

bcs_status axpby(Solver* s, double a, const double* x, double b, double* y, size_t N) {
  BCS_LAUNCH(s, K_BLAS, 24.0 * N, 3.0 * N, k_axpby, vgrid(N), 256, 0, a, x, b, y, N);
  return BCS_OK;
}

bcs_status scale_copy(Solver* s, double a, const double* x, double* y, size_t N) {
  BCS_LAUNCH(s, K_BLAS, 16.0 * N, 1.0 * N, k_scale, vgrid(N), 256, 0, a, x, y, N);
  return BCS_OK;
}

bcs_status bicg_p_update(Solver* s, double beta, double omega, const double* r, const double* v, double* p,
                         size_t N) {
  BCS_LAUNCH(s, K_BLAS, 32.0 * N, 4.0 * N, k_bicg_p, vgrid(N), 256, 0, beta, omega, r, v, p, N);
  return BCS_OK;
}


}  // namespace bcs
