// Device prefix sums and per-segment sort/unique used by the structure and
// setup phases (row pointers, sparsity patterns of Galerkin products).
#include <algorithm>
#include <climits>

#include "internal.h"

namespace bcs {

namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Block-local exclusive scan of one tile; writes the tile total.
__global__ void k_scan_tile(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                            int32_t* __restrict__ tile_sum, int n) {
  dep_enter();
  __shared__ int32_t warp_tot[SCAN_THREADS / 32];
  const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  int32_t v[SCAN_ITEMS];
  int32_t local = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int i = base + k;
    v[k] = i < n ? in[i] : 0;
    local += v[k];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t incl = local;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int32_t w = lane < SCAN_THREADS / 32 ? warp_tot[lane] : 0;
    int32_t wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t t = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += t;
    }
    if (lane < SCAN_THREADS / 32) warp_tot[lane] = wi - w;  // exclusive warp offsets
    if (lane == SCAN_THREADS / 32 - 1) tile_sum[blockIdx.x] = wi;
  }
  __syncthreads();
  int32_t run = warp_tot[warp] + incl - local;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int i = base + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
}

// out[i] += tile_off[i / SCAN_TILE]; thread n writes the grand total.
__global__ void k_scan_add(int32_t* __restrict__ out, const int32_t* __restrict__ tile_off, int n, int tiles) {
  dep_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += tile_off[i / SCAN_TILE];
  else if (i == n) out[n] = tile_off[tiles];
}

// Whole exclusive scan of n <= SMALL_SCAN_MAX values in one block, total to
// out[n]. Values move through shared memory with coalesced global loads and
// stores; each thread scans SMALL_ITEMS consecutive values (row index padded
// by one word per 32 so those reads are free of bank conflicts).
constexpr int SMALL_THREADS = 1024;
constexpr int SMALL_ITEMS = 8;
constexpr int SMALL_SCAN_MAX = SMALL_THREADS * SMALL_ITEMS;

__device__ __forceinline__ int pad32(int i) { return i + (i >> 5); }

__global__ void __launch_bounds__(SMALL_THREADS) k_scan_small(const int32_t* __restrict__ in,
                                                             int32_t* __restrict__ out, int n) {
  dep_enter();
  __shared__ int32_t buf[SMALL_SCAN_MAX + SMALL_SCAN_MAX / 32];
  __shared__ int32_t warp_tot[SMALL_THREADS / 32];
#pragma unroll
  for (int k = 0; k < SMALL_ITEMS; ++k) {
    const int i = k * SMALL_THREADS + threadIdx.x;
    buf[pad32(i)] = i < n ? in[i] : 0;
  }
  __syncthreads();
  const int base = threadIdx.x * SMALL_ITEMS;
  int32_t v[SMALL_ITEMS];
  int32_t local = 0;
#pragma unroll
  for (int k = 0; k < SMALL_ITEMS; ++k) {
    v[k] = buf[pad32(base + k)];
    local += v[k];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t incl = local;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int32_t w = warp_tot[lane];
    int32_t wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t t = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += t;
    }
    warp_tot[lane] = wi - w;
    if (lane == 31) out[n] = wi;
  }
  __syncthreads();
  int32_t run = warp_tot[warp] + incl - local;
#pragma unroll
  for (int k = 0; k < SMALL_ITEMS; ++k) {
    buf[pad32(base + k)] = run;
    run += v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < SMALL_ITEMS; ++k) {
    const int i = k * SMALL_THREADS + threadIdx.x;
    if (i < n) out[i] = buf[pad32(i)];
  }
}

}  // namespace

// out[0..n) = exclusive prefix sums of in[0..n), out[n] = the total; in and
// out must not overlap. One launch up to SMALL_SCAN_MAX values, else tiles of
// SCAN_TILE, a scan of the tile sums and an add pass.
bcs_status exclusive_scan(Solver* s, const int32_t* in, int32_t* out, int n) {
  if (n <= 0) {
    BCS_CU(s, cudaMemsetAsync(out, 0, sizeof(int32_t), s->stream));
    return BCS_OK;
  }
  if (n <= SMALL_SCAN_MAX) {
    BCS_LAUNCH_DEP(s, K_MISC, 8.0 * n, 0, k_scan_small, 1, SMALL_THREADS, 0, in, out, n);
    return BCS_OK;
  }
  const int tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  DBuf<int32_t> sums, offs;
  BCS_ALLOC(s, sums, tiles);
  BCS_ALLOC(s, offs, tiles + 1);
  BCS_LAUNCH_DEP(s, K_MISC, 8.0 * n, 0, k_scan_tile, tiles, SCAN_THREADS, 0, in, out, sums.p, n);
  BCS_OKR(exclusive_scan(s, sums.p, offs.p, tiles));
  BCS_LAUNCH_DEP(s, K_MISC, 8.0 * n, 0, k_scan_add, grid_for((size_t)n + 1, 256), 256, 0, out, offs.p, n, tiles);
  return BCS_OK;
}

// ------------------------------------------------------------------ sort/unique
// Per-segment ascending sort of int32 keys with duplicates removed (counts
// written), or of uint64 keys kept whole (sort only). Segments up to 32 keys:
// one thread (register insertion network); up to 256: one warp (bitonic in
// shared memory); longer: one block per segment (bitonic in dynamic shared
// memory).
namespace {

constexpr int WARP_SEG_MAX = 256;  // segments up to this length: one warp
constexpr int WARPS_PER_BLOCK = 4;
constexpr int BLOCK_SEG_MAX = 16384;

template <class T> __device__ __forceinline__ T key_max();
template <> __device__ __forceinline__ int32_t key_max<int32_t>() { return INT_MAX; }
template <> __device__ __forceinline__ uint64_t key_max<uint64_t>() { return ~0ull; }

// One warp per row of list[0 .. *n_list) (rows longer than 32 keys), grid-
// stride over the list; rows longer than WARP_SEG_MAX go to long_rows.
template <class T, bool UNIQUE>
__global__ void k_seg_sort_warp(const int32_t* __restrict__ seg_ptr, T* __restrict__ keys,
                                int32_t* __restrict__ count, const int32_t* __restrict__ list,
                                const int32_t* __restrict__ n_list, int32_t* __restrict__ long_rows,
                                int32_t* __restrict__ n_long) {
  dep_enter();
  __shared__ T sm[WARPS_PER_BLOCK][WARP_SEG_MAX];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nl = *n_list;
  for (int idx = blockIdx.x * WARPS_PER_BLOCK + warp; idx < nl; idx += gridDim.x * WARPS_PER_BLOCK) {
    const int r = list[idx];
    const int b = seg_ptr[r], len = seg_ptr[r + 1] - b;
    if (len > WARP_SEG_MAX) {
      if (lane == 0) long_rows[atomicAdd(n_long, 1)] = r;
      continue;
    }
    if (len <= 64) {
      // register bitonic sort of 64 slots: lane l holds elements l and l + 32
      T a0 = lane < len ? keys[b + lane] : key_max<T>();
      T a1 = lane + 32 < len ? keys[b + 32 + lane] : key_max<T>();
      for (int k = 2; k <= 64; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
          if (j == 32) {  // k == 64: elements l and l + 32, ascending
            const T lo = a0 < a1 ? a0 : a1, hi = a0 < a1 ? a1 : a0;
            a0 = lo;
            a1 = hi;
          } else {
            const T p0 = __shfl_xor_sync(0xffffffffu, a0, j), p1 = __shfl_xor_sync(0xffffffffu, a1, j);
            const bool lower = (lane & j) == 0;
            const bool up0 = (lane & k) == 0, up1 = ((lane + 32) & k) == 0;
            a0 = (lower == up0) ? (p0 < a0 ? p0 : a0) : (p0 < a0 ? a0 : p0);
            a1 = (lower == up1) ? (p1 < a1 ? p1 : a1) : (p1 < a1 ? a1 : p1);
          }
        }
      if (!UNIQUE) {
        if (lane < len) keys[b + lane] = a0;
        if (lane + 32 < len) keys[b + 32 + lane] = a1;
        continue;
      }
      const T prev0 = __shfl_up_sync(0xffffffffu, a0, 1);
      const T last0 = __shfl_sync(0xffffffffu, a0, 31);
      const T up1v = __shfl_up_sync(0xffffffffu, a1, 1);
      const T prev1 = lane == 0 ? last0 : up1v;
      const bool keep0 = lane < len && (lane == 0 || a0 != prev0);
      const bool keep1 = lane + 32 < len && a1 != prev1;
      const unsigned m0 = __ballot_sync(0xffffffffu, keep0), m1 = __ballot_sync(0xffffffffu, keep1);
      const unsigned below = (1u << lane) - 1u;
      if (keep0) keys[b + __popc(m0 & below)] = a0;
      if (keep1) keys[b + __popc(m0) + __popc(m1 & below)] = a1;
      if (lane == 0) count[r] = __popc(m0) + __popc(m1);
      continue;
    }
    T* a = sm[warp];
    int S = 32;
    while (S < len) S <<= 1;
    for (int i = lane; i < S; i += 32) a[i] = i < len ? keys[b + i] : key_max<T>();
    __syncwarp();
    for (int k = 2; k <= S; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = lane; i < S; i += 32) {
          const int l = i ^ j;
          if (l > i) {
            const T x = a[i], y = a[l];
            const bool up = (i & k) == 0;
            if ((x > y) == up) {
              a[i] = y;
              a[l] = x;
            }
          }
        }
        __syncwarp();
      }
    if (!UNIQUE) {
      for (int i = lane; i < len; i += 32) keys[b + i] = a[i];
      __syncwarp();
      continue;
    }
    int outpos = 0;
    for (int i0 = 0; i0 < len; i0 += 32) {
      const int i = i0 + lane;
      const bool keep = i < len && (i == 0 || a[i] != a[i - 1]);
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) keys[b + outpos + __popc(m & ((1u << lane) - 1u))] = a[i];
      outpos += __popc(m);
    }
    if (lane == 0) count[r] = outpos;
    __syncwarp();
  }
}

template <class T, bool UNIQUE>
__global__ void k_seg_sort_block(const int32_t* __restrict__ seg_ptr, T* __restrict__ keys,
                                 int32_t* __restrict__ count, const int32_t* __restrict__ long_rows) {
  dep_enter();
  extern __shared__ __align__(16) unsigned char dyn[];
  T* a = reinterpret_cast<T*>(dyn);
  __shared__ int32_t wsum[32];
  const int r = long_rows[blockIdx.x];
  const int b = seg_ptr[r], len = seg_ptr[r + 1] - b;
  int S = 32;
  while (S < len) S <<= 1;
  for (int i = threadIdx.x; i < S; i += blockDim.x) a[i] = i < len ? keys[b + i] : key_max<T>();
  __syncthreads();
  for (int k = 2; k <= S; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < S; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const T x = a[i], y = a[l];
          const bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncthreads();
    }
  if (!UNIQUE) {
    for (int i = threadIdx.x; i < len; i += blockDim.x) keys[b + i] = a[i];
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int base = 0;
  for (int i0 = 0; i0 < len; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    const bool keep = i < len && (i == 0 || a[i] != a[i - 1]);
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) wsum[warp] = __popc(m);
    __syncthreads();
    int off = base, tot = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) off += wsum[w];
      tot += wsum[w];
    }
    if (keep) keys[b + off + __popc(m & ((1u << lane) - 1u))] = a[i];
    base += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) count[r] = base;
}

// Segments of at most M keys: one thread sorts its segment in registers
// (an unrolled insertion network of min/max pairs).
template <int M, class T, bool UNIQUE>
__global__ void k_seg_sort_thread(const int32_t* __restrict__ seg_ptr, T* __restrict__ keys,
                                  int32_t* __restrict__ count, int rows, int32_t* __restrict__ defer,
                                  int32_t* __restrict__ n_defer) {
  dep_enter();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int b = seg_ptr[r], len = seg_ptr[r + 1] - b;
  if (len > M) {  // longer rows (only present when defer is given) go to the warp kernel
    defer[atomicAdd(n_defer, 1)] = r;
    return;
  }
  T a[M];
#pragma unroll
  for (int i = 0; i < M; ++i) a[i] = i < len ? keys[b + i] : key_max<T>();
#pragma unroll
  for (int i = 1; i < M; ++i)
#pragma unroll
    for (int j = i; j > 0; --j) {
      const T lo = min(a[j - 1], a[j]), hi = max(a[j - 1], a[j]);
      a[j - 1] = lo;
      a[j] = hi;
    }
  if (!UNIQUE) {
#pragma unroll
    for (int i = 0; i < M; ++i)
      if (i < len) keys[b + i] = a[i];
    return;
  }
  int out = 0;
#pragma unroll
  for (int i = 0; i < M; ++i)
    if (i < len && (i == 0 || a[i] != a[i - 1])) keys[b + out++] = a[i];
  count[r] = out;
}

template <class T, bool UNIQUE>
bcs_status seg_sort(Solver* s, const int32_t* seg_ptr, T* keys, int32_t* count, int rows, int max_len) {
  if (rows <= 0) return BCS_OK;
  if (max_len > BLOCK_SEG_MAX)
    return s->fail(BCS_EINVAL, "a sparsity-pattern row has more than 16384 candidate entries");
  if (max_len <= 16) {
    BCS_LAUNCH_DEP(s, K_MISC, 0, 0, (k_seg_sort_thread<16, T, UNIQUE>), grid_for(rows, 128), 128, 0, seg_ptr, keys,
               count, rows, (int32_t*)nullptr, (int32_t*)nullptr);
    return BCS_OK;
  }
  if (max_len <= 32) {
    BCS_LAUNCH_DEP(s, K_MISC, 0, 0, (k_seg_sort_thread<32, T, UNIQUE>), grid_for(rows, 128), 128, 0, seg_ptr, keys,
               count, rows, (int32_t*)nullptr, (int32_t*)nullptr);
    return BCS_OK;
  }
  // rows of up to 32 keys by one thread each; longer rows listed for one
  // warp each; rows beyond WARP_SEG_MAX listed again for one block each
  DBuf<int32_t> mid_rows, long_rows, aux;
  BCS_ALLOC(s, mid_rows, rows);
  BCS_ALLOC(s, long_rows, rows);
  BCS_ALLOC(s, aux, 2);
  BCS_CU(s, cudaMemsetAsync(aux.p, 0, 2 * sizeof(int32_t), s->stream));
  BCS_LAUNCH_DEP(s, K_MISC, 0, 0, (k_seg_sort_thread<32, T, UNIQUE>), grid_for(rows, 128), 128, 0, seg_ptr, keys, count,
             rows, mid_rows.p, aux.p);
  const unsigned gw = std::min<unsigned>(grid_for(rows, WARPS_PER_BLOCK), 2048u);
  BCS_LAUNCH_DEP(s, K_MISC, 0, 0, (k_seg_sort_warp<T, UNIQUE>), gw, 32 * WARPS_PER_BLOCK, 0, seg_ptr, keys, count,
             mid_rows.p, aux.p, long_rows.p, aux.p + 1);
  if (max_len > WARP_SEG_MAX) {
    int32_t h = 0;
    BCS_CU(s, cudaMemcpyAsync(&h, aux.p + 1, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
    BCS_CU(s, cudaStreamSynchronize(s->stream));
    if (h > 0) {
      int S = 32;
      while (S < max_len) S <<= 1;
      const size_t smem = (size_t)S * sizeof(T);
      constexpr auto kseg = k_seg_sort_block<T, UNIQUE>;
      BCS_CU(s, allow_max_dynamic_smem<kseg>());
      BCS_LAUNCH_DEP(s, K_MISC, 0, 0, (k_seg_sort_block<T, UNIQUE>), h, 512, smem, seg_ptr, keys, count, long_rows.p);
    }
  }
  return BCS_OK;
}

}  // namespace

bcs_status segmented_sort_unique(Solver* s, const int32_t* seg_ptr, int32_t* keys, int32_t* count,
                                 int rows, int max_len) {
  return seg_sort<int32_t, true>(s, seg_ptr, keys, count, rows, max_len);
}

bcs_status segmented_sort64(Solver* s, const int32_t* seg_ptr, uint64_t* keys, int rows, int max_len) {
  return seg_sort<uint64_t, false>(s, seg_ptr, keys, nullptr, rows, max_len);
}

}  // namespace bcs
