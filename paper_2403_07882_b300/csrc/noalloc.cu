// LDU face addressing -> block-CSR structure without any device allocation.
//
// Some callers cannot let a library allocate device memory: host programs
// that reserve the GPU's memory up front and run under a hard budget, and
// applications that forbid cudaMalloc/cudaFree after start-up because those
// calls synchronise the device and stall every other stream. For them,
// bcs_ldu_structure_noalloc() builds the same structure as bcs_set_structure
// into caller-provided device arrays, keeping its scratch (per-row cursors,
// scan tile sums, error flags) in the fixed array below.
//
// The scratch is a file-scope __device__ array, so every GPU that loads this
// library holds it (about 4 MB) until the process exits. Every call shares
// it and it keeps the last call's contents; the kernels clear what must start
// at zero. Calls that overlap on the GPU (for example on two streams at once)
// race on this scratch and must be serialised by the caller.
#include <cstdio>
#include <mutex>

#include "internal.h"

namespace {

constexpr int NA_MAX_CELLS = 1 << 20;                       // 1,048,576 cells
constexpr int NA_TILE = 1024;                               // scan tile (one block)
constexpr int NA_MAX_TILES = NA_MAX_CELLS / NA_TILE;        // 1024
constexpr int NA_FLAGS = 8;
constexpr int NA_SCRATCH_INTS = NA_MAX_CELLS + NA_MAX_TILES + NA_FLAGS;

// cursor[NA_MAX_CELLS] | tile sums[NA_MAX_TILES] | flags[NA_FLAGS]
static __device__ __align__(256) int32_t g_na_scratch[NA_SCRATCH_INTS];

// Device addresses of g_na_scratch, one per device, filled on the first call
// made with that device current. In host code the symbol itself is only a
// host-side stand-in, never a device address. The cached address belongs to
// the device's primary context as it stood at that first call: it does not
// survive a reset of that context (cudaDeviceReset), after which this entry
// point must not be called again in the same process.
std::mutex g_na_mutex;
int32_t* g_na_ptr[256] = {};

__global__ void k_na_init(int C, int32_t* __restrict__ cnt, int32_t* __restrict__ cursor,
                          int32_t* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < C) {
    cnt[i] = 1;      // the diagonal block
    cursor[i] = 1;   // faces go after the diagonal
  }
  if (i == 0) flag[0] = 0;
}

__global__ void k_na_count(int C, int F, const int32_t* __restrict__ owner, const int32_t* __restrict__ nb,
                           int32_t* __restrict__ cnt, int32_t* __restrict__ flag) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const int o = owner[f], m = nb[f];
  if (o < 0 || o >= C || m < 0 || m >= C || o == m) {
    atomicOr(flag, 1);
    return;
  }
  atomicAdd(&cnt[o], 1);
  atomicAdd(&cnt[m], 1);
}

// In-place exclusive scan of one 1024-element tile; tile total to tiles[].
__global__ void __launch_bounds__(NA_TILE) k_na_scan_tile(int C, int32_t* __restrict__ a,
                                                          int32_t* __restrict__ tiles) {
  __shared__ int32_t wsum[32];
  const int i = blockIdx.x * NA_TILE + threadIdx.x;
  const int v = i < C ? a[i] : 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += t;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int w = wsum[lane];
    int wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += t;
    }
    wsum[lane] = wi - w;
    if (lane == 31) tiles[blockIdx.x] = wi;
  }
  __syncthreads();
  if (i < C) a[i] = wsum[warp] + incl - v;
}

// Exclusive scan of the tile sums (one block); the grand total goes to a[C].
__global__ void __launch_bounds__(NA_TILE) k_na_scan_tiles(int ntiles, int32_t* __restrict__ tiles,
                                                           int32_t* __restrict__ a, int C) {
  __shared__ int32_t wsum[32];
  const int t = threadIdx.x;
  const int v = t < ntiles ? tiles[t] : 0;
  const int lane = t & 31, warp = t >> 5;
  int incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += u;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int w = wsum[lane];
    int wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += u;
    }
    wsum[lane] = wi - w;
    if (lane == 31) a[C] = wi;
  }
  __syncthreads();
  if (t < ntiles) tiles[t] = wsum[warp] + incl - v;
}

__global__ void k_na_scan_add(int C, int32_t* __restrict__ a, const int32_t* __restrict__ tiles) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < C) a[i] += tiles[i / NA_TILE];
}

// The kernels after the face check skip their work when it failed (flag bit
// 1), so a bad face never indexes the output arrays and the host reads the
// flag once, at the end.
__global__ void k_na_place(int C, int F, const int32_t* __restrict__ owner, const int32_t* __restrict__ nb,
                           const int32_t* __restrict__ rp, int32_t* __restrict__ cursor, int32_t* __restrict__ col,
                           const int32_t* __restrict__ flag) {
  if (*flag & 1) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < C) col[rp[t]] = t;
  if (t < F) {
    const int o = owner[t], m = nb[t];
    col[rp[o] + atomicAdd(&cursor[o], 1)] = m;
    col[rp[m] + atomicAdd(&cursor[m], 1)] = o;
  }
}

__global__ void k_na_sort(int C, const int32_t* __restrict__ rp, int32_t* __restrict__ col, int32_t* flag) {
  if (*flag & 1) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C) return;
  const int b = rp[i], e = rp[i + 1];
  for (int p = b + 1; p < e; ++p) {
    const int c = col[p];
    int q = p - 1;
    while (q >= b && col[q] > c) {
      col[q + 1] = col[q];
      --q;
    }
    col[q + 1] = c;
  }
  for (int p = b + 1; p < e; ++p)
    if (col[p] == col[p - 1]) atomicOr(flag, 2);
}

__device__ __forceinline__ int na_find(const int32_t* __restrict__ col, int b, int e, int j) {
  while (b < e) {
    const int m = (b + e) >> 1;
    if (col[m] == j) return m;
    if (col[m] < j) b = m + 1;
    else e = m;
  }
  return -1;
}

__global__ void k_na_positions(int C, int F, const int32_t* __restrict__ owner, const int32_t* __restrict__ nb,
                               const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                               int32_t* __restrict__ pos_diag, int32_t* __restrict__ pos_up,
                               int32_t* __restrict__ pos_lo, const int32_t* __restrict__ flag) {
  if (*flag & 1) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < C) pos_diag[t] = na_find(col, rp[t], rp[t + 1], t);
  if (t < F) {
    const int o = owner[t], m = nb[t];
    pos_up[t] = na_find(col, rp[o], rp[o + 1], m);
    pos_lo[t] = na_find(col, rp[m], rp[m + 1], o);
  }
}

bcs_status na_fail(char* err, size_t len, bcs_status st, const char* msg) {
  if (err && len) std::snprintf(err, len, "%s", msg);
  return st;
}

#define NA_CU(call)                                                                          \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      if (err && errlen) std::snprintf(err, errlen, "%s: %s", #call, cudaGetErrorString(e_)); \
      return BCS_ECUDA;                                                                      \
    }                                                                                        \
  } while (0)

}  // namespace

extern "C" BCS_API bcs_status bcs_ldu_structure_noalloc(int32_t C, int32_t F, const int32_t* owner,
                                                        const int32_t* neighbour, int32_t* row_ptr, int32_t* col,
                                                        int32_t* pos_diag, int32_t* pos_up, int32_t* pos_lo,
                                                        void* stream, char* err, size_t errlen) {
  if (err && errlen) err[0] = '\0';
  if (C < 1 || F < 0) return na_fail(err, errlen, BCS_EINVAL, "n_cells must be >= 1 and n_faces >= 0");
  if (C > NA_MAX_CELLS)
    return na_fail(err, errlen, BCS_EINVAL,
                   "n_cells exceeds the 1048576-cell limit of the allocation-free structure build");
  if ((long long)C + 2LL * F > (long long)INT32_MAX / 64)
    return na_fail(err, errlen, BCS_EINVAL, "too many blocks for int32 indexing");
  if (!row_ptr || !col || !pos_diag || (F > 0 && (!owner || !neighbour || !pos_up || !pos_lo)))
    return na_fail(err, errlen, BCS_EINVAL, "null array argument");
  int dev = 0;
  NA_CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return na_fail(err, errlen, BCS_EINVAL, "device ordinal out of range");
  // every array must be device memory of the current device: a host pointer
  // handed to the kernels would be dereferenced on the GPU
  {
    const void* arrays[7] = {owner, neighbour, row_ptr, col, pos_diag, pos_up, pos_lo};
    for (const void* a : arrays) {
      if (!a) continue;
      cudaPointerAttributes at{};
      const cudaError_t e = cudaPointerGetAttributes(&at, a);
      if (e != cudaSuccess) {
        (void)cudaGetLastError();  // clear the error this query leaves behind
        return na_fail(err, errlen, BCS_EINVAL, "an array is not device memory");
      }
      if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev)
        return na_fail(err, errlen, BCS_EINVAL, "an array is not device memory of the current device");
    }
  }
  int32_t* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      void* p = nullptr;
      NA_CU(cudaGetSymbolAddress(&p, g_na_scratch));
      g_na_ptr[dev] = static_cast<int32_t*>(p);
    }
    scratch = g_na_ptr[dev];
  }
  int32_t* cursor = scratch;
  int32_t* tiles = scratch + NA_MAX_CELLS;
  int32_t* flag = tiles + NA_MAX_TILES;
  cudaStream_t st = (cudaStream_t)stream;
  const int CF = C > F ? C : F;
  const int ntiles = (C + NA_TILE - 1) / NA_TILE;
  k_na_init<<<bcs::grid_for(C, 256), 256, 0, st>>>(C, row_ptr, cursor, flag);
  if (F > 0) k_na_count<<<bcs::grid_for(F, 256), 256, 0, st>>>(C, F, owner, neighbour, row_ptr, flag);
  k_na_scan_tile<<<ntiles, NA_TILE, 0, st>>>(C, row_ptr, tiles);
  k_na_scan_tiles<<<1, NA_TILE, 0, st>>>(ntiles, tiles, row_ptr, C);
  k_na_scan_add<<<bcs::grid_for(C, 256), 256, 0, st>>>(C, row_ptr, tiles);
  k_na_place<<<bcs::grid_for(CF, 256), 256, 0, st>>>(C, F, owner, neighbour, row_ptr, cursor, col, flag);
  k_na_sort<<<bcs::grid_for(C, 128), 128, 0, st>>>(C, row_ptr, col, flag);
  k_na_positions<<<bcs::grid_for(CF, 256), 256, 0, st>>>(C, F, owner, neighbour, row_ptr, col, pos_diag, pos_up,
                                                          pos_lo, flag);
  NA_CU(cudaGetLastError());
  // pinned staging of the flag is not available without allocating, so the
  // read goes to pageable host memory and completes before the sync returns
  int32_t h = 0;
  NA_CU(cudaMemcpyAsync(&h, flag, sizeof(h), cudaMemcpyDeviceToHost, st));
  NA_CU(cudaStreamSynchronize(st));
  if (h & 1) return na_fail(err, errlen, BCS_EINVAL, "face addressing: cell id out of range or owner == neighbour");
  if (h & 2) return na_fail(err, errlen, BCS_EINVAL, "face addressing: a face (cell pair) is repeated");
  return BCS_OK;
}
