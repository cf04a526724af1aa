// Register-resident Gauss-Jordan inverse of one N x N block per thread
// (block-Jacobi inverses, DILU factor). Device code shared by setup.cu and
// dilu.cu; both need the same operation order so that every FP64 inverse
// equals the CPU reference bit for bit.
#pragma once
#include <utility>

namespace bcs {

// Gauss-Jordan inverse of one N x N block per thread: implicit partial
// pivoting (largest |M[r][k]| among unused rows, first on ties), one
// reciprocal per pivot, l = M[r][k] * (1 / pivot), updates
// M[r][j] = fma(-l, M[p][j], M[r][j]) for j >= k, deferred normalisation
// inv[k][:] = M[p_k][N:] * (1 / M[p_k][k]). Steps are unrolled at compile
// time and the pivot row is picked with bit masks, so M stays in registers.
// T = double (the FP64 inverses the oracle reproduces) or float (the FP32
// inverses of the FP32 / BF16 block-Jacobi smoother).
template <class T>
struct GjBits;
template <>
struct GjBits<double> {
  using I = long long;
  __device__ static I bits(double v) { return __double_as_longlong(v); }
  __device__ static double val(I b) { return __longlong_as_double(b); }
};
template <>
struct GjBits<float> {
  using I = int;
  __device__ static I bits(float v) { return __float_as_int(v); }
  __device__ static float val(I b) { return __int_as_float(b); }
};

template <class T>
__device__ __forceinline__ T pick(T v, bool on) {
  using B = GjBits<T>;
  return B::val(B::bits(v) & ((typename B::I)0 - (typename B::I)on));
}

template <int N, class T = double>
struct BlockGJ {
  using B = GjBits<T>;
  T M[N][2 * N];
  unsigned used = 0;
  int prow[N];
  bool bad = false;

  template <int K>
  __device__ __forceinline__ void step() {
    int p = 0;
    T best = -1;
#pragma unroll
    for (int r = 0; r < N; ++r) {
      const T v = fabs(M[r][K]);
      const bool take = !(used & (1u << r)) && v > best;
      best = take ? v : best;
      p = take ? r : p;
    }
    T pr[2 * N];
#pragma unroll
    for (int j = K; j < 2 * N; ++j) {
      typename B::I t = 0;
#pragma unroll
      for (int r = 0; r < N; ++r) t |= B::bits(pick(M[r][j], p == r));
      pr[j] = B::val(t);
    }
    bad |= pr[K] == (T)0;
    used |= 1u << p;
    prow[K] = p;
    const T rpiv = (T)1 / pr[K];
#pragma unroll
    for (int r = 0; r < N; ++r) {
      const T l = M[r][K] * rpiv;
#pragma unroll
      for (int j = K; j < 2 * N; ++j) {
        const T nv = fma(-l, pr[j], M[r][j]);
        M[r][j] = B::val(B::bits(pick(M[r][j], r == p)) | B::bits(pick(nv, r != p)));
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
template <int N, class T>
__device__ __forceinline__ bool gj_finish(BlockGJ<N, T>& g, T* __restrict__ o) {
  using B = GjBits<T>;
#pragma unroll
  for (int r = 0; r < N; ++r)
#pragma unroll
    for (int c = 0; c < N; ++c) g.M[r][N + c] = r == c ? (T)1 : (T)0;
  g.run(std::make_integer_sequence<int, N>{});
  if (g.bad) return false;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    T pr[2 * N];
#pragma unroll
    for (int j = 0; j < 2 * N; ++j) {
      typename B::I t = 0;
#pragma unroll
      for (int r = 0; r < N; ++r) t |= B::bits(pick(g.M[r][j], g.prow[k] == r));
      pr[j] = B::val(t);
    }
    const T rd = (T)1 / pr[k];
#pragma unroll
    for (int j = 0; j < N; ++j) o[k * N + j] = pr[N + j] * rd;
  }
  return true;
}

}  // namespace bcs
