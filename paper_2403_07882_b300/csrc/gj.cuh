// Register-resident Gauss-Jordan inverse of one N x N FP64 block per thread
// (block-Jacobi inverses, DILU factor). Device code shared by setup.cu and
// dilu.cu; both need the same operation order so that every inverse equals
// the CPU reference bit for bit.
#pragma once
#include <utility>

namespace bcs {

// Gauss-Jordan inverse of one N x N block per thread: implicit partial
// pivoting (largest |M[r][k]| among unused rows, first on ties), one
// reciprocal per pivot, l = M[r][k] * (1 / pivot), updates
// M[r][j] = fma(-l, M[p][j], M[r][j]) for j >= k, deferred normalisation
// inv[k][:] = M[p_k][N:] * (1 / M[p_k][k]). Steps are unrolled at compile
// time and the pivot row is picked with bit masks, so M stays in registers.
__device__ __forceinline__ double pick(double v, bool on) {
  return __longlong_as_double(__double_as_longlong(v) & (0ll - (long long)on));
}

template <int N>
struct BlockGJ {
  double M[N][2 * N];
  unsigned used = 0;
  int prow[N];
  bool bad = false;

  template <int K>
  __device__ __forceinline__ void step() {
    int p = 0;
    double best = -1.0;
#pragma unroll
    for (int r = 0; r < N; ++r) {
      const double v = fabs(M[r][K]);
      const bool take = !(used & (1u << r)) && v > best;
      best = take ? v : best;
      p = take ? r : p;
    }
    double pr[2 * N];
#pragma unroll
    for (int j = K; j < 2 * N; ++j) {
      long long t = 0;
#pragma unroll
      for (int r = 0; r < N; ++r) t |= __double_as_longlong(pick(M[r][j], p == r));
      pr[j] = __longlong_as_double(t);
    }
    bad |= pr[K] == 0.0;
    used |= 1u << p;
    prow[K] = p;
    const double rpiv = 1.0 / pr[K];
#pragma unroll
    for (int r = 0; r < N; ++r) {
      const double l = M[r][K] * rpiv;
#pragma unroll
      for (int j = K; j < 2 * N; ++j) {
        const double nv = fma(-l, pr[j], M[r][j]);
        M[r][j] = __longlong_as_double(__double_as_longlong(pick(M[r][j], r == p)) |
                                       __double_as_longlong(pick(nv, r != p)));
      }
    }
  }
  template <int... K>
  __device__ __forceinline__ void run(std::integer_sequence<int, K...>) {
    (step<K>(), ...);
  }
};


// Load M's left half first (g.M[r][c], c < N), then call finish(out): sets
// the right half to I, eliminates, writes the inverse to out (row-major).
// Returns false (out untouched) when a pivot is exactly zero.
template <int N>
__device__ __forceinline__ bool gj_finish(BlockGJ<N>& g, double* __restrict__ o) {
#pragma unroll
  for (int r = 0; r < N; ++r)
#pragma unroll
    for (int c = 0; c < N; ++c) g.M[r][N + c] = r == c ? 1.0 : 0.0;
  g.run(std::make_integer_sequence<int, N>{});
  if (g.bad) return false;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    double pr[2 * N];
#pragma unroll
    for (int j = 0; j < 2 * N; ++j) {
      long long t = 0;
#pragma unroll
      for (int r = 0; r < N; ++r) t |= __double_as_longlong(pick(g.M[r][j], g.prow[k] == r));
      pr[j] = __longlong_as_double(t);
    }
    const double rd = 1.0 / pr[k];
#pragma unroll
    for (int j = 0; j < N; ++j) o[k * N + j] = pr[N + j] * rd;
  }
  return true;
}

}  // namespace bcs
