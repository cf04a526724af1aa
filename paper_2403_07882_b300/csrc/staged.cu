// Block-Jacobi sweep and residual of the FP32 / BF16 V-cycle with per-warp
// bulk-copy (TMA) staging of block rows.
//
// The block rows of a warp tile (floor(32 / n) consecutive rows) occupy one
// contiguous span of the value array and one of the column array. Lane 0 of
// each warp copies the next tile's two spans into shared memory with
// cp.async.bulk (16-byte aligned: the span is widened to 16-byte boundaries,
// buffers carry 16 bytes of tail padding) completing on an mbarrier, while
// the warp computes the current tile from the other buffer. HBM is thus read
// in long sequential bursts without occupying the load/store units, and the
// lanes read their block-row entries from shared memory (lane l: scalar row
// l % n of block row l / n). Waits are bounded: a wait that gives up sets an
// error bit that the solve reports as BCS_TIMEOUT.
#include "internal.h"

namespace bcs {

namespace {

constexpr int ST_WARPS = 8;
constexpr int ST_MAX_SMEM = 200 * 1024;
constexpr int ST_WAIT_LIMIT = 1 << 22;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ float ldv(const float* p) { return *p; }
__device__ __forceinline__ float ldv(const bf16* p) { return __bfloat162float(*p); }

__host__ __device__ constexpr size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

// JACOBI: y = x + omega D^-1 (b - A x); otherwise y = b - A x.
template <int N, class TV, bool JACOBI>
__global__ void __launch_bounds__(ST_WARPS * 32) k_staged(int rows, int ntiles, const int32_t* __restrict__ rp,
                                                          const int32_t* __restrict__ ci, const TV* __restrict__ val,
                                                          const float* __restrict__ dinv, const float* __restrict__ x,
                                                          const float* __restrict__ b, float* __restrict__ y,
                                                          float omega, int vcap, int ccap,
                                                          int32_t* __restrict__ err) {
  constexpr int RPW = 32 / N, NN = N * N;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[ST_WARPS][2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int stage_bytes = vcap + ccap;
  unsigned char* wbase = smem + (size_t)warp * 2 * stage_bytes;
  uint64_t* bar = bars[warp];
  if (lane == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    fence_mbar_init();
  }
  __syncwarp();
  const int rw = lane / N, r = lane - rw * N;
  const int gwarp = blockIdx.x * ST_WARPS + warp, nwarps = gridDim.x * ST_WARPS;

  auto issue = [&](int t, int stg) {
    const int i0 = t * RPW, i1 = min(i0 + RPW, rows);
    const size_t kb = (size_t)rp[i0], ke = (size_t)rp[i1];
    const size_t vs = kb * NN * sizeof(TV) & ~(size_t)15, ve = align16(ke * NN * sizeof(TV));
    const size_t cs = kb * 4 & ~(size_t)15, ce = align16(ke * 4);
    unsigned char* st = wbase + (size_t)stg * stage_bytes;
    fence_proxy_async();
    mbar_expect_tx(&bar[stg], (uint32_t)((ve - vs) + (ce - cs)));
    bulk_g2s(st, (const unsigned char*)val + vs, (uint32_t)(ve - vs), &bar[stg]);
    bulk_g2s(st + vcap, (const unsigned char*)ci + cs, (uint32_t)(ce - cs), &bar[stg]);
  };

  uint32_t phase = 0;
  int stg = 0;
  int t = gwarp;
  if (t < ntiles && lane == 0) issue(t, 0);
  for (; t < ntiles; t += nwarps) {
    const int tn = t + nwarps;
    if (tn < ntiles && lane == 0) issue(tn, stg ^ 1);
    bool ok = false;
    for (int it = 0; it < ST_WAIT_LIMIT; ++it)
      if (mbar_try_wait(&bar[stg], (phase >> stg) & 1u)) {
        ok = true;
        break;
      }
    if (!ok) {
      if (lane == 0) atomicOr(err, 32);
      return;
    }
    phase ^= 1u << stg;
    const int i0 = t * RPW;
    const size_t kb = (size_t)rp[i0];
    const unsigned char* st = wbase + (size_t)stg * stage_bytes;
    const TV* sv = (const TV*)(st + ((kb * NN * sizeof(TV)) & 15));
    const int32_t* sc = (const int32_t*)(st + vcap + ((kb * 4) & 15));
    const int i = i0 + rw;
    const bool active = rw < RPW && i < rows;
    float acc = 0.f;
    if (active) {
      const int a0 = rp[i] - (int)kb, a1 = rp[i + 1] - (int)kb;
      for (int k = a0; k < a1; ++k) {
        const int j = sc[k];
        const TV* a = sv + (size_t)k * NN + r * N;
        const float* xj = x + (size_t)j * N;
#pragma unroll
        for (int c = 0; c < N; ++c) acc = fmaf(ldv(a + c), __ldg(xj + c), acc);
      }
    }
    if (JACOBI) {
      const float res = active ? b[(size_t)i * N + r] - acc : 0.f;
      float tt = 0.f;
#pragma unroll
      for (int c = 0; c < N; ++c) {
        const float rc = __shfl_sync(0xffffffffu, res, (rw * N + c) & 31);
        if (active) tt = fmaf(__ldg(dinv + ((size_t)i * N + r) * N + c), rc, tt);
      }
      if (active) y[(size_t)i * N + r] = x[(size_t)i * N + r] + omega * tt;
    } else if (active) {
      y[(size_t)i * N + r] = b[(size_t)i * N + r] - acc;
    }
    __syncwarp();
    stg ^= 1;
  }
}

__global__ void k_tile_max(int rows, int rpw, const int32_t* __restrict__ rp, int32_t* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i0 = t * rpw;
  if (i0 >= rows) return;
  const int i1 = min(i0 + rpw, rows);
  atomicMax(out, rp[i1] - rp[i0]);
}

struct Plan {
  int vcap, ccap, smem, blocks, ntiles;
};

template <int N, class TV, bool JACOBI>
bool make_plan(Solver* s, const Level& L, Plan* p) {
  if (L.max_tile_blocks <= 0) return false;
  constexpr int NN = N * N;
  p->vcap = (int)(align16((size_t)L.max_tile_blocks * NN * sizeof(TV)) + 16);
  p->ccap = (int)(align16((size_t)L.max_tile_blocks * 4) + 16);
  p->smem = ST_WARPS * 2 * (p->vcap + p->ccap);
  if (p->smem > ST_MAX_SMEM) return false;
  static int configured_smem = 0;  // per instantiation
  if (p->smem > configured_smem) {
    if (cudaFuncSetAttribute(k_staged<N, TV, JACOBI>, cudaFuncAttributeMaxDynamicSharedMemorySize, ST_MAX_SMEM) !=
        cudaSuccess) {
      (void)cudaGetLastError();
      return false;
    }
    configured_smem = ST_MAX_SMEM;
  }
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_staged<N, TV, JACOBI>, ST_WARPS * 32, p->smem) !=
          cudaSuccess ||
      per_sm < 1) {
    (void)cudaGetLastError();
    return false;
  }
  constexpr int RPW = 32 / N;
  p->ntiles = (L.A.rows + RPW - 1) / RPW;
  const int want = (p->ntiles + ST_WARPS - 1) / ST_WARPS;
  p->blocks = want < sms * per_sm ? want : sms * per_sm;
  return true;
}

}  // namespace

bcs_status level_tile_stats(Solver* s, Level& L) {
  if (L.max_tile_blocks >= 0) return BCS_OK;
  const int rpw = 32 / s->n;
  const int ntiles = (L.A.rows + rpw - 1) / rpw;
  DBuf<int32_t> m;
  BCS_ALLOC(s, m, 1);
  BCS_CU(s, cudaMemsetAsync(m.p, 0, sizeof(int32_t), s->stream));
  BCS_LAUNCH(s, K_MISC, 0, 0, k_tile_max, grid_for(ntiles, 256), 256, 0, L.A.rows, rpw, L.A.rp.p, m.p);
  int32_t h = 0;
  BCS_CU(s, cudaMemcpyAsync(&h, m.p, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  L.max_tile_blocks = h;
  return BCS_OK;
}

template <int N, class TV>
bcs_status staged_sweep(Solver* s, Level& L, const TV* val, const float* dinv, const float* x, const float* b,
                        float* y, float omega, bool* used) {
  Plan p;
  *used = make_plan<N, TV, true>(s, L, &p);
  if (!*used) return BCS_OK;
  const int rows = L.A.rows;
  const double bytes = (double)L.A.nnz * (N * N * sizeof(TV) + 4) + 4.0 * (rows + 1) +
                       (double)rows * N * (N * sizeof(float) + 3 * sizeof(float));
  BCS_LAUNCH(s, K_SWEEP, bytes, 2.0 * (L.A.nnz + rows) * N * N, (k_staged<N, TV, true>), p.blocks, ST_WARPS * 32,
             p.smem, rows, p.ntiles, L.A.rp.p, L.A.ci.p, val, dinv, x, b, y, omega, p.vcap, p.ccap, s->flag.p + 1);
  return BCS_OK;
}

template <int N, class TV>
bcs_status staged_resid(Solver* s, Level& L, const TV* val, const float* x, const float* b, float* r, bool* used) {
  Plan p;
  *used = make_plan<N, TV, false>(s, L, &p);
  if (!*used) return BCS_OK;
  const int rows = L.A.rows;
  const double bytes = (double)L.A.nnz * (N * N * sizeof(TV) + 4) + 4.0 * (rows + 1) + (double)rows * N * 3 * 4;
  BCS_LAUNCH(s, K_RESID, bytes, 2.0 * L.A.nnz * N * N, (k_staged<N, TV, false>), p.blocks, ST_WARPS * 32, p.smem,
             rows, p.ntiles, L.A.rp.p, L.A.ci.p, val, (const float*)nullptr, x, b, r, 0.f, p.vcap, p.ccap,
             s->flag.p + 1);
  return BCS_OK;
}

#define BCS_STAGED_INST(N)                                                                                      \
  template bcs_status staged_sweep<N, float>(Solver*, Level&, const float*, const float*, const float*,        \
                                             const float*, float*, float, bool*);                              \
  template bcs_status staged_sweep<N, bf16>(Solver*, Level&, const bf16*, const float*, const float*,          \
                                            const float*, float*, float, bool*);                               \
  template bcs_status staged_resid<N, float>(Solver*, Level&, const float*, const float*, const float*, float*, \
                                             bool*);                                                           \
  template bcs_status staged_resid<N, bf16>(Solver*, Level&, const bf16*, const float*, const float*, float*,  \
                                            bool*);
BCS_STAGED_INST(1)
BCS_STAGED_INST(2)
BCS_STAGED_INST(3)
BCS_STAGED_INST(4)
BCS_STAGED_INST(5)
BCS_STAGED_INST(6)
BCS_STAGED_INST(7)
BCS_STAGED_INST(8)

}  // namespace bcs
