// Internal declarations of the block-coupled solver library (not installed).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/bcs.h"

namespace bcs {

using bf16 = __nv_bfloat16;

// NVTX range over a library call (header-only NVTX 3: a no-op unless a
// profiler such as Nsight attaches its tool).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Kernel kinds for launch counting and event timing.
enum Kind {
  K_CONVERT = 0,    // LDU -> BSR structure / value permutation
  K_SPMV64 = 1,     // FP64 outer SpMV / true residual
  K_SWEEP = 2,      // block-Jacobi sweep (SpMV + D^-1 epilogue)
  K_RESID = 3,      // V-cycle residual
  K_TRANSFER = 4,   // restriction / prolongation
  K_COARSE = 5,     // coarsest-level solve
  K_BLAS = 6,       // dots, norms, axpy, Gram-Schmidt
  K_SETUP_AGG = 7,  // strength, matching, numbering
  K_SETUP_GAL = 8,  // Galerkin products, prolongation
  K_SETUP_INV = 9,  // block inverses, coarse inverse
  K_CAST = 10,      // precision casts
  K_MISC = 11,      // scans, sorts
  K_TUNE = 12,      // layout autotuning launches
  K_ASSEMBLE = 13,  // assembly of the density-based system
  K_NKINDS = 14
};
const char* kind_name(int k);

// ------------------------------------------------------------ device memory
// Stream-ordered allocations (cudaMallocAsync) on the solver's stream.
struct Alloc {
  cudaStream_t stream = nullptr;
  size_t live = 0;
  // caller's allocator (bcs_config.alloc / release), else cudaMallocAsync
  void* (*fa)(size_t, void*, void*) = nullptr;
  void (*fr)(void*, size_t, void*, void*) = nullptr;
  void* user = nullptr;
  void* get(size_t bytes);
  void put(void* p, size_t bytes);
};

template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  Alloc* a = nullptr;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept { *this = std::move(o); }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p;
      n = o.n;
      a = o.a;
      o.p = nullptr;
      o.n = 0;
    }
    return *this;
  }
  ~DBuf() { release(); }
  void release() {
    if (p && a) a->put(p, n * sizeof(T));
    p = nullptr;
    n = 0;
  }
  // (Re)allocates when the size differs; contents undefined. False on OOM.
  bool resize(Alloc* al, size_t count) {
    if (count == n && (p || count == 0)) return true;
    release();
    a = al;
    if (count == 0) return true;
    p = static_cast<T*>(al->get(count * sizeof(T)));
    if (!p) return false;
    n = count;
    return true;
  }
};

// Step tile of the thread-per-block-row sliced layout (layout 1, cycle.cu):
// 32 block rows' n*n entries; entry e of slice lane w sits in 16-byte groups
// of G consecutive entries (group g of lane w at g * G * 32 + w * G), the
// n*n mod G remaining entries element-major after the groups.
template <int NN, class TV>
struct TprTile {
  static constexpr int G = 16 / (int)sizeof(TV);  // entries per 16-byte group
  static constexpr int NG = NN / G;               // full groups
  static constexpr int R = NN - NG * G;           // remaining entries
  static constexpr int TILE = NN * 32;
  __host__ __device__ static constexpr int off(int e, int w) {
    return e < NG * G ? (e / G) * G * 32 + w * G + e % G : NG * G * 32 + (e - NG * G) * 32 + w;
  }
};

// ----------------------------------------------------------- data structures
// Block-CSR matrix on the device; values FP64 (setup precision).
struct Bsr {
  int rows = 0, cols = 0, nnz = 0;
  int maxrow = -1;  // longest row (blocks), -1 when not known
  DBuf<int32_t> rp, ci;
  DBuf<double> v;
};

// Plan of the tentative Galerkin product: per coarse row I its terms
// sk[seg[I] .. seg[I+1]) sorted by (output block, fine position): the fine
// block position of each, the first term of every output block flagged by
// the sign bit (outputs follow in the row's column order).
struct TentPlan {
  DBuf<int32_t> seg, sk;
};

struct Level {
  Bsr A;                     // FP64 operator of this level
  DBuf<int32_t> dpos;        // diagonal block position per row
  DBuf<double> dinv;         // FP64 diagonal block inverses (when dinv64)
  DBuf<float> dinv32;        // FP32 block inverses for the FP32 / BF16 cycle
  // dinv holds this setup's FP64 inverses; false when the setup inverted the
  // blocks in FP32 straight into dinv32 (FP32 / BF16 block-Jacobi cycle)
  bool dinv64 = true;
  // transfer to level l+1 (absent at the coarsest level)
  int nagg = 0;
  DBuf<int32_t> agg;         // aggregate of each row
  DBuf<int32_t> mptr, mem;   // aggregate member lists (members ascending)
  DBuf<int32_t> cnt;         // member counts (between aggregation and the member lists)
  int maxmem = 0;            // largest aggregate (an upper bound)
  Bsr P, R, AP;              // smoothed mode only: P, R and the product A P (FP64)
  DBuf<int32_t> Prow, Rrow, AProw, Crow;  // row of every nonzero of P, R, AP, A_{l+1}
  TentPlan tent;              // plan of the tentative Galerkin product
  DBuf<float> P32, R32;
  DBuf<bf16> P16, R16;
  double omega_p = 0.0;
  int coarse_kind = -1;      // -1 not coarsest, 0 dense inverse, 1 sweeps
  // sliced copy of A for the FP32 / BF16 cycle: slices of consecutive block
  // rows; slice s covers steps sptr[s] .. sptr[s+1]; step t holds one block per
  // row (padding past a row's end)
  // layout (smap): 0 = one lane per scalar row, floor(32/n) block rows per
  // warp; 1 = one thread per block row, 32 block rows per warp; -1 = not
  // chosen yet (picked by the layout autotuner at full setup)
  int smap = -1;
  int nslices = 0, nsteps = 0;
  DBuf<int32_t> sptr, sci;
  DBuf<int32_t> srow;        // layout 1: block row at each slice position
  // layout 1 of the fine level: the slot (step * 32 + slice lane) of every
  // block-CSR position, recorded by the first fill; through it the value
  // gather of a later upload writes the sliced copy itself
  DBuf<int32_t> tpos;
  DBuf<float> s32;
  DBuf<bf16> s16;
  DBuf<char> vx, vb, vr, vt; // V-cycle vectors (cycle precision)
  // multicolour block DILU smoother (smoother = 1); ncol = -1: block Jacobi
  int ncol = -1;
  DBuf<int32_t> colour;      // colour of each row
  DBuf<int32_t> crow;        // rows grouped by colour: cstart[c] .. cstart[c+1]
  std::vector<int> cstart;
  DBuf<int32_t> cstart_d;    // cstart on the device
  int dcl = 0;               // FP32 / BF16 cycle: blocks of the one-launch DILU step's cluster (0: per colour)
  DBuf<double> einv;         // E_i^{-1}, FP64 (when einv64)
  // einv holds this setup's FP64 factor; false when the DILU factor of the
  // FP32 / BF16 cycle was computed in FP32 straight into einv32
  bool einv64 = true;
  // each row's off-diagonal blocks split for the sweeps: the lower part
  // (colour(j) < colour(i)) then the upper part (colour(j) > colour(i)),
  // each in column order, stored in colour-list order: the row at crow[t]
  // at [dptr[t], dptr[t+1]), lower part ending at dmid[t]; dsrc: BSR
  // position, dci: column (built with the colouring)
  DBuf<int32_t> dptr, dmid, dsrc, dci;
  DBuf<float> einv32, a32;   // FP32 copies for the FP32 / BF16 cycle (a32: split-order values)
  DBuf<bf16> a16;            // BF16 split-order values for the BF16 cycle
  DBuf<char> vd;             // DILU correction vector (cycle precision)
};

// Coarse tail of the V-cycle (the levels below a size threshold) run as one
// thread-block-cluster launch: a list of phases over a table of levels and a
// table of vectors (ids 0 and 1: the tail's own right-hand side and
// solution, passed at launch).
enum TailOp { T_JAC0 = 0, T_SWEEP, T_RESID, T_RESTRICT, T_PROLONG, T_GEMV, T_ZERO };
struct TailPhase {
  int op, level;   // level: index into the tail's level table
  int ia, ib, iy;  // vector ids: input x (or r, x_c), right-hand side b, output
};
struct TailLevel {
  int rows, nslices, nagg, pad;
  const int32_t *rp, *sptr, *sci, *mptr, *mem, *agg;
  const void* sv;       // sliced values (lane-per-row layout), FP32 or BF16
  const float* dinv;    // FP32 block inverses
};
struct TailPlan {
  int nph = 0, cluster = 0;
  size_t level_off = 0, vec_off = 0;
  double bytes = 0.0, flops = 0.0;
  DBuf<char> buf;  // phases | levels | vector pointers
};

// FGMRES restart cycle kept on the device (restart length m <= KS_MAXM): the
// Arnoldi step index, the rotated Hessenberg matrix, the Givens rotations,
// the rotated right-hand side g and the stop decision, so that a cycle runs
// without reading anything back to the host.
constexpr int KS_MAXM = 64;
struct KrylovState {
  int j;        // Arnoldi step of the cycle being computed
  int iters;    // iterations of the whole solve so far
  int stop;     // KS_RUN or why the cycle ended
  int jend;     // steps completed in this cycle
  int m, maxiter;
  double tol, bnorm, rhn;  // rhn = 1 / h_{j+1,j} of the last step
  double g[KS_MAXM + 1], cs[KS_MAXM], sn[KS_MAXM], y[KS_MAXM];
  double H[(KS_MAXM + 1) * KS_MAXM];  // row-major, leading dimension m
};
enum { KS_RUN = 0, KS_CONVERGED = 1, KS_HAPPY = 2, KS_BREAKDOWN = 3, KS_MAXITER = 4, KS_CYCLE_END = 5 };

// BiCGStab iteration kept on the device: its scalars and why the loop left
// (an event the host acts on: breakdown restart, a small residual to
// confirm on the true residual, the iteration limit).
struct BicgState {
  int it, stop, first, maxiter;
  double tol, bnorm, rho, rho_old, alpha, omega, beta;
};
enum { BS_RUN = 0, BS_BREAK = 1, BS_S_SMALL = 2, BS_R_SMALL = 3, BS_OMEGA0 = 4, BS_MAXITER = 5 };

// Device scalar slots of the Krylov solvers (s->scal): first and second
// Gram-Schmidt pass, norms, the nonzero flag of x0, a restart cycle's
// outcome (iterations, steps, stop reason).
constexpr int SLOT_A = 0, SLOT_B = 72, SLOT_N = 144, SLOT_X = 145, SLOT_S = 146;

// Batched solves: several systems' FGMRES run in lockstep, each step's
// kernels covering every case (blockIdx.z = case) through these tables.
constexpr int BATCH_MAX_LEVELS = 20;
struct BLevel {  // one level of one case's hierarchy (FP32 / BF16 cycle)
  int rows, nslices, smap, nagg, coarse_kind, pad;
  const int32_t *rp, *srow, *sptr, *sci, *mptr, *mem, *agg;
  const void* sv;      // sliced values in the level's layout
  const float* dinv;   // FP32 block inverses
  float *vb, *vx, *vr, *vt;
};
struct BCase {
  int n_levels, rows;
  size_t N;                       // unknowns
  KrylovState* ks;
  int* live;                      // this step's participation (set at the step's start)
  const int* round;               // 1 while the case takes part in the current restart round
  double *V, *w, *kt, *scal, *red, *x, *r;
  const double* b;
  float* Z;
  const int32_t *rp, *ci;         // fine FP64 matrix
  const double* val;
  const double* cinv;
  int cN, pad;
  BLevel lv[BATCH_MAX_LEVELS];
};

struct Timer {
  int kind;
  cudaEvent_t a, b;
  const char* what;
  double bytes;
  int level;  // hierarchy level the launch works on (-1: none)
};

// Per-level totals of the timed launches (profile = 1), by kernel kind.
constexpr int LEVEL_TIMES_MAX = 64;
struct LevelTime {
  long long launches[BCS_NUM_KERNEL_KINDS] = {};
  double ms[BCS_NUM_KERNEL_KINDS] = {};
  double bytes[BCS_NUM_KERNEL_KINDS] = {};
};

struct NamedTime {
  long long launches = 0;
  double ms = 0.0, bytes = 0.0;
  int kind = -1;
};

struct Solver {
  int n = 0;
  bcs_config cfg{};
  bcs_config setup_cfg{};        // options the hierarchy was built with
  cudaStream_t stream = nullptr;
  Alloc alloc;
  std::string err;
  // structure
  int C = 0, F = 0, nnz = 0;
  bool have_structure = false, have_values = false, have_hierarchy = false;
  DBuf<int32_t> src;             // BSR position -> LDU source code
  DBuf<int32_t> pos_diag, pos_up, pos_lo;
  // locality reorder (cfg.reorder): internal row i is the caller's cell
  // perm[i], inv[cell] = i; pos_diag and the diagonal source codes stay in
  // the caller's numbering
  bool reordered = false;
  DBuf<int32_t> perm, inv;
  DBuf<double> rb, rx;           // vectors in the internal numbering
  DBuf<double> stage_d, stage_u, stage_l;  // host-input staging
  // block Frobenius norms of the fine matrix, computed by the value gather
  // when a full setup follows (fresh: they belong to the current values)
  DBuf<double> nrm0;
  bool nrm0_fresh = false;
  // precision of the fine level's sliced copy when the value gather wrote
  // it through lv[0].tpos (the copy then skips its fill), else -1; set by
  // the gather, cleared when the new values have been set up
  int v0_direct = -1;
  cudaStream_t cstream = nullptr;          // host -> device copies of the values in pieces
  cudaStream_t sstream = nullptr;          // setup work beside the aggregation (block inverses)
  cudaEvent_t sev[2] = {};
  std::vector<cudaEvent_t> copy_events;     // one per piece
  DBuf<int32_t> stage_o, stage_n;
  // hierarchy
  std::vector<Level> lv;
  DBuf<double> cinv;             // coarsest dense inverse (FP64)
  int cN = 0;
  // Krylov work space
  DBuf<double> kv;               // FGMRES V (m+1 vectors) / BiCGStab vectors
  DBuf<char> kz;                 // FGMRES Z (m vectors, cycle precision)
  DBuf<double> kw, kr, kx, kb, kt;  // kt: FP64 copy of an FP32 preconditioned vector
  DBuf<double> red;              // reduction partials
  DBuf<double> scal;             // device scalars
  double* hscal = nullptr;       // pinned host mirror of scal
  DBuf<int32_t> flag;            // device status flags
  // statistics
  long long launches = 0;
  long long kind_launches[BCS_NUM_KERNEL_KINDS] = {};
  double kind_bytes[BCS_NUM_KERNEL_KINDS] = {};
  double kind_flops[BCS_NUM_KERNEL_KINDS] = {};
  double kind_ms[BCS_NUM_KERNEL_KINDS] = {};
  std::vector<Timer> timers;
  std::map<std::string, NamedTime> named;  // per kernel name (profile = 1)
  // Level the launches being issued work on (set by the setup's level loop,
  // the FP32 copies and the V-cycle; -1 outside them) and the per-level
  // totals of the timed launches.
  int cur_level = -1;
  std::vector<LevelTime> level_times;
  std::vector<cudaEvent_t> event_pool;
  size_t event_next = 0;
  double last_setup_ms = 0.0;
  long long host_syncs = 0;      // scalar reads that waited for the device (solves)
  // V-cycle captured as a CUDA graph (FP32 / BF16 cycle): input lv[0].vb,
  // output lv[0].vx; dropped at every setup / resetup and on destroy
  cudaGraphExec_t cyc_exec = nullptr;
  int tail_level = -1;             // first level of the coarse tail (-1: none)
  TailPlan tail;
  cudaStream_t gstream = nullptr;  // private stream the graph is captured on
  long long cyc_kind_launches[BCS_NUM_KERNEL_KINDS] = {};
  double cyc_kind_bytes[BCS_NUM_KERNEL_KINDS] = {}, cyc_kind_flops[BCS_NUM_KERNEL_KINDS] = {};
  // FGMRES Arnoldi steps replayed as one graph with a device-side loop exit
  // (a conditional WHILE node); body launches counted per executed step
  cudaGraphExec_t kry_exec = nullptr;
  long long kry_kind_launches[BCS_NUM_KERNEL_KINDS] = {};
  double kry_kind_bytes[BCS_NUM_KERNEL_KINDS] = {}, kry_kind_flops[BCS_NUM_KERNEL_KINDS] = {};
  DBuf<char> kst;                // KrylovState / BicgState
  cudaGraphExec_t bcg_exec = nullptr;  // BiCGStab iteration in a graph WHILE node
  const void* bcg_key[3] = {};
  double* kx_dev = nullptr;            // the solution vector the captured BiCGStab step updates
  long long bcg_kind_launches[BCS_NUM_KERNEL_KINDS] = {};
  double bcg_kind_bytes[BCS_NUM_KERNEL_KINDS] = {}, bcg_kind_flops[BCS_NUM_KERNEL_KINDS] = {};
  const void* kry_key[5] = {};    // buffers the captured step uses (recapture when one moves)
  int kry_m = 0;
  DBuf<double> kvj, kzj;         // FP64 cycle: fixed input / output of the preconditioner
  void drop_graph() {
    if (cyc_exec) cudaGraphExecDestroy(cyc_exec);
    cyc_exec = nullptr;
    if (kry_exec) cudaGraphExecDestroy(kry_exec);
    kry_exec = nullptr;
    if (bcg_exec) cudaGraphExecDestroy(bcg_exec);
    bcg_exec = nullptr;
  }

  bcs_status fail(bcs_status st, const std::string& m) {
    err = m;
    return st;
  }
  void pre(int kind);
  bcs_status post(int kind, const char* what, double bytes, double flops);
  void flush_timers();
};

// Sets s->cur_level for the lifetime of the guard and restores the previous
// value after it.
struct LevelScope {
  Solver* s;
  int prev;
  LevelScope(Solver* s_, int l) : s(s_), prev(s_->cur_level) { s->cur_level = l; }
  ~LevelScope() { s->cur_level = prev; }
};

// A failed call also clears the thread's last-error state, so that no later
// launch check reports it as its own.
#define BCS_CU(S, call)                                                                  \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      (void)cudaGetLastError();                                                          \
      return (S)->fail(BCS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    }                                                                                    \
  } while (0)
#define BCS_OKR(...)                \
  do {                              \
    bcs_status st_ = (__VA_ARGS__); \
    if (st_ != BCS_OK) return st_;  \
  } while (0)
#define BCS_ALLOC(S, buf, count)                                                        \
  do {                                                                                  \
    if (!(buf).resize(&(S)->alloc, (count)))                                            \
      return (S)->fail(BCS_ENOMEM, std::string("device allocation failed: ") + #buf);   \
  } while (0)

// Programmatic dependent launch (sm_90 and later). A kernel launched with
// BCS_LAUNCH_DEP may be scheduled while its predecessor in the stream is
// still finishing; it calls dep_enter() first, which waits for that grid to
// complete with its memory visible before the kernel reads or writes any
// data, then lets the kernel's own successor begin launching. Launched
// without the attribute, both instructions return at once.
__device__ __forceinline__ void dep_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The dynamic shared-memory limit of a kernel is state of the process, not
// of a launch: raising it to the device's opt-in maximum (less the kernel's
// static shared memory) once, thread-safe,
// lets every launch ask for what it needs without racing other threads that
// set the limit for their own launches.
template <auto kernel>
cudaError_t allow_max_dynamic_smem() {
  static std::once_flag once;  // one per kernel
  static cudaError_t result = cudaSuccess;
  std::call_once(once, [&] {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    result = cudaGetDevice(&dev);
    if (result == cudaSuccess) result = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (result == cudaSuccess) result = cudaFuncGetAttributes(&fa, kernel);
    // the limit covers the dynamic part; the kernel's static shared memory
    // counts against the same per-block maximum
    if (result == cudaSuccess)
      result = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    optin - (int)fa.sharedSizeBytes);
    if (result != cudaSuccess) (void)cudaGetLastError();
  });
  return result;
}

// BCS_LAUNCH with the programmatic-serialization attribute (when
// cfg.dependent_launch is set); the kernel must begin with dep_enter(). A
// failed launch clears the thread's last-error state, so that no later
// launch reports it as its own.
#define BCS_LAUNCH_DEP(S, KIND, BYTES, FLOPS, kernel, grid, block, smem, ...)                       \
  do {                                                                                              \
    (S)->pre(KIND);                                                                                 \
    cudaLaunchConfig_t lc_{};                                                                       \
    cudaLaunchAttribute at_[1];                                                                     \
    at_[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;                                 \
    at_[0].val.programmaticStreamSerializationAllowed = 1;                                          \
    lc_.gridDim = dim3(grid);                                                                       \
    lc_.blockDim = dim3(block);                                                                     \
    lc_.dynamicSmemBytes = (smem);                                                                  \
    lc_.stream = (S)->stream;                                                                       \
    lc_.attrs = at_;                                                                                \
    lc_.numAttrs = (S)->cfg.dependent_launch ? 1 : 0;                                               \
    const cudaError_t le_ = cudaLaunchKernelEx(&lc_, kernel, __VA_ARGS__);                          \
    if (le_ != cudaSuccess) {                                                                       \
      (void)cudaGetLastError();                                                                     \
      return (S)->fail(BCS_ECUDA, std::string(#kernel) + ": " + cudaGetErrorString(le_));           \
    }                                                                                               \
    bcs_status st_ = (S)->post(KIND, #kernel, (BYTES), (FLOPS));                                    \
    if (st_ != BCS_OK) return st_;                                                                  \
  } while (0)

// Launch kernel<<<grid, block, smem, s->stream>>>(args...) with bookkeeping.
#define BCS_LAUNCH(S, KIND, BYTES, FLOPS, kernel, grid, block, smem, ...)  \
  do {                                                                    \
    (S)->pre(KIND);                                                       \
    kernel<<<(grid), (block), (smem), (S)->stream>>>(__VA_ARGS__);         \
    bcs_status st_ = (S)->post(KIND, #kernel, (BYTES), (FLOPS));          \
    if (st_ != BCS_OK) return st_;                                        \
  } while (0)

inline unsigned grid_for(size_t work, int block) {
  size_t g = (work + block - 1) / block;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// Block-size dispatch: calls f(std::integral_constant<int, N>) for n = 1..8.
template <class F>
bcs_status with_n(int n, F&& f) {
  switch (n) {
    case 1: return f(std::integral_constant<int, 1>{});
    case 2: return f(std::integral_constant<int, 2>{});
    case 3: return f(std::integral_constant<int, 3>{});
    case 4: return f(std::integral_constant<int, 4>{});
    case 5: return f(std::integral_constant<int, 5>{});
    case 6: return f(std::integral_constant<int, 6>{});
    case 7: return f(std::integral_constant<int, 7>{});
    case 8: return f(std::integral_constant<int, 8>{});
    default: return BCS_EINVAL;
  }
}

// ------------------------------------------------------------------ format.cu
bcs_status build_structure(Solver* s, const int32_t* owner_d, const int32_t* nb_d);
// reorder.cu: reverse Cuthill-McKee order of A's rows (perm[new] = old,
// inv[old] = new) and its application
bcs_status rcm_order(Solver* s, const Bsr& A, int32_t* perm, int32_t* inv);
bcs_status relabel_faces(Solver* s, const int32_t* o, const int32_t* nb, int32_t* o2, int32_t* nb2);
bcs_status user_diag_maps(Solver* s);
bcs_status to_internal(Solver* s, const double* user, double* internal);  // [C][n] vectors
bcs_status to_user(Solver* s, const double* internal, double* user);
// pack.cu: segregated fields <-> block AoS (at most PK_MAX_FIELDS fields);
// src of pack_coefficients: 3 pointers (diag, upper, lower) per (row field,
// column field) pair, nullptr = zero coupling; diag == nullptr writes the fine
// block-CSR values
constexpr int PK_MAX_FIELDS = 8;
bcs_status pack_vector(Solver* s, int nfields, const int* ncomp, const double* const* fields, double* out);
bcs_status unpack_vector(Solver* s, int nfields, const int* ncomp, const double* in, double* const* fields);
bcs_status pack_coefficients(Solver* s, int nfields, const int* ncomp, const double* const* src, double* diag,
                             double* upper, double* lower);
// assemble.cu: density-based system from cell states and face geometry;
// diag == nullptr writes the fine block-CSR values, else the LDU arrays
bcs_status assemble_density(Solver* s, const double* Q, const double* area, const double* normal, const double* dist,
                            const bcs_flow_params& prm, double* diag, double* upper, double* lower);
bcs_status permute_values(Solver* s, const double* diag_d, const double* upper_d,
                          const double* lower_d);
// The same from HOST arrays, the copy overlapped with the scatter.
bcs_status upload_values(Solver* s, const double* diag_h, const double* upper_h, const double* lower_h);

// -------------------------------------------------------------------- scan.cu
// out[0..n] = exclusive prefix sums of in[0..n-1]; out[n] = total. Device.
bcs_status exclusive_scan(Solver* s, const int32_t* in, int32_t* out, int n);
// Per-segment sort + unique of int keys: seg_ptr[rows+1] delimits segments of
// keys; on return count[r] holds the unique count of segment r and the
// segment starts with its sorted unique keys. max_len bounds the segments.
bcs_status segmented_sort_unique(Solver* s, const int32_t* seg_ptr, int32_t* keys,
                                 int32_t* count, int rows, int max_len);
// Ascending sort of every segment of 64-bit keys (duplicates kept).
bcs_status segmented_sort64(Solver* s, const int32_t* seg_ptr, uint64_t* keys, int rows, int max_len);

// -------------------------------------------------------------------- blas.cu
// Deterministic FP64 reductions into s->scal[slot...].
bcs_status dot(Solver* s, const double* x, const double* y, size_t N, int slot);
bcs_status multidot(Solver* s, const double* V, size_t ldv, int k, const double* w, size_t N,
                    int slot);
bcs_status fetch_scalars(Solver* s, int count);  // scal[0..count) -> hscal, synchronises
// scal[slot] = 1.0 if any x[i] != 0, else 0.0 (no sync)
bcs_status any_nonzero(Solver* s, const double* x, size_t N, int slot);
bcs_status axpby(Solver* s, double a, const double* x, double b, double* y, size_t N);
bcs_status scale_copy(Solver* s, double a, const double* x, double* y, size_t N);
bcs_status gs_update(Solver* s, const double* V, size_t ldv, int k, const double* hdev, double* w,
                     size_t N);
bcs_status add_combination(Solver* s, const void* Z, bool z_float, size_t ldz, int k,
                           const double* ydev, double* x, size_t N);
bcs_status bicg_p_update(Solver* s, double beta, double omega, const double* r, const double* v,
                         double* p, size_t N);
// Gram-Schmidt pass 2 fused with the norm: w -= sum_{q<k} h[q] V_q, then
// scal[slot] = ||w||^2 with the reduction tree of dot() (same bits).
bcs_status gs_update_norm(Solver* s, const double* V, size_t ldv, int k, const double* hdev, double* w, size_t N,
                          int slot);
// Steps of the device-resident FGMRES cycle; ks is the KrylovState in device
// memory, the step index j is read from it.
bcs_status ks_init(Solver* s, KrylovState* ks, double beta, double bnorm, int iters, int m, int maxiter,
                   double tol);
bcs_status ks_take_vj(Solver* s, const double* V, size_t ldv, const KrylovState* ks, void* out, bool to_float,
                      size_t N);
bcs_status ks_store_z(Solver* s, const void* zsrc, bool z_float, void* Z, const KrylovState* ks, double* widen,
                      size_t N);
bcs_status ks_multidot(Solver* s, const double* V, size_t ldv, const KrylovState* ks, const double* w, bool with_w,
                       size_t N, int slot);
bcs_status ks_gs_update(Solver* s, const double* V, size_t ldv, const KrylovState* ks, const double* hdev, double* w,
                        size_t N, int norm_slot);
bcs_status ks_givens(Solver* s, KrylovState* ks, int slot_a, int slot_b, int slot_n,
                     cudaGraphConditionalHandle cond);
bcs_status ks_scale_next(Solver* s, const KrylovState* ks, const double* w, double* V, size_t ldv, size_t N);
bcs_status ks_finish_cycle(Solver* s, KrylovState* ks, const void* Z, bool z_float, double* x, size_t N);
bcs_status ks_export(Solver* s, const KrylovState* ks, int slot);
// BiCGStab on the device (state bs; scalars from s->scal)
bcs_status bs_init(Solver* s, BicgState* bs, int it, int maxiter, double tol, double bnorm, int first);
bcs_status bs_rho(Solver* s, BicgState* bs);
bcs_status bs_p_update(Solver* s, const BicgState* bs, const double* r, const double* v, double* p, size_t N);
bcs_status bs_alpha(Solver* s, BicgState* bs);
bcs_status bs_s_update(Solver* s, const BicgState* bs, const double* r, const double* v, double* sv, size_t N);
bcs_status bs_snorm(Solver* s, BicgState* bs);
bcs_status bs_omega(Solver* s, BicgState* bs);
bcs_status bs_x_update(Solver* s, const BicgState* bs, const void* ph, bool z_float, double* x, size_t N);
bcs_status bs_r_update(Solver* s, const BicgState* bs, const double* sv, const double* t, double* r, size_t N);
bcs_status bs_end(Solver* s, BicgState* bs, cudaGraphConditionalHandle cond);
bcs_status bs_export(Solver* s, const BicgState* bs);  // it, stop, alpha -> scal[SLOT_S ..]
// Batched steps (launched on s's stream; cases is a device table of count
// entries; kmax bounds the vectors of one multi-dot, rows / N the largest
// case).
bcs_status kb_step_begin(Solver* s, const BCase* cases, int count);
bcs_status kb_take_vj(Solver* s, const BCase* cases, int count, size_t maxN);
bcs_status kb_store_z(Solver* s, const BCase* cases, int count, size_t maxN);
bcs_status kb_multidot(Solver* s, const BCase* cases, int count, bool with_w, int kmax, int slot);
bcs_status kb_gs_update(Solver* s, const BCase* cases, int count, int hslot, int nslot);
bcs_status kb_givens(Solver* s, const BCase* cases, int count, cudaGraphConditionalHandle cond);
bcs_status kb_scale_next(Solver* s, const BCase* cases, int count, size_t maxN);
bcs_status kb_finish(Solver* s, const BCase* cases, int count, size_t maxN);
bcs_status kb_norm_r(Solver* s, const BCase* cases, int count);
bcs_status kb_gather_out(Solver* s, const BCase* cases, int count, double* out);
// cycle.cu: the batched V-cycle (level-0 vb -> vx of every live case) and
// the FP64 products of the batched step
bcs_status kb_cycle(Solver* s, const BCase* cases, const std::vector<BCase>& host, int count);
bcs_status kb_spmv_w(Solver* s, const BCase* cases, int count, int max_rows);
bcs_status kb_resid_r(Solver* s, const BCase* cases, int count, int max_rows);

// ------------------------------------------------------------------- cycle.cu
enum Mode { M_SPMV = 0, M_ADD = 1, M_RESID = 2 };
// y = A x (b == nullptr) or y = b - A x with the FP64 matrix; x double or float.
bcs_status spmv64(Solver* s, const Bsr& A, const void* x, bool x_is_float, double* y,
                  const double* b, int kind);
// keep_graphs: a values-only resetup (every buffer kept in place), so the
// captured graphs stay valid; otherwise they are dropped.
bcs_status cycle_prepare(Solver* s, bool keep_graphs = false);
// Where the value gather writes the fine level's sliced copy: the slot map
// and the buffer of the precision the next setup uses (one of s32, s16
// set), or all null when it cannot: no slot map yet (the first setup of a
// structure fills the copy and records it), another layout or precision,
// an unsliced cycle. The buffer is never allocated here: allocated before
// a full setup (which then runs with it held), the copy made every later
// full setup of a 2.1 M block-row structure about 3 ms slower with the
// same kernel times (measured; the cause was not isolated), so a new
// structure's first setup fills the copy after the hierarchy is built.
struct SliceTarget {
  const int32_t* tpos = nullptr;
  float* s32 = nullptr;
  bf16* s16 = nullptr;
  int prec = -1;
};
bcs_status fine_slice_target(Solver* s, SliceTarget* t);
// The blocks' FP64 inverses of level l into out (computed on demand when the
// setup inverted them in FP32 only).
bcs_status level_dinv64(Solver* s, int l, const double** out, DBuf<double>& tmp);
// Whether the setup inverts the diagonal blocks in FP32 only (an FP32 / BF16
// cycle whose configuration reads no FP64 inverses).
bool fp32_inverses(const Solver* s);
// The DILU factor's FP64 inverses E_i^{-1} of level l into out (computed on
// demand when the setup built the FP32 factor only).
bcs_status dilu_einv64(Solver* s, int l, const double** out, DBuf<double>& tmp);
bcs_status precond_apply(Solver* s, const double* v, void* z);  // z in cycle precision
bcs_status jacobi_apply(Solver* s, const double* v, double* z);
bcs_status sgs_apply(Solver* s, const double* v, void* z);  // z in cycle precision
// The preconditioners between fixed buffers, launched kernel by kernel (for
// capture into a larger graph): the FP64 V-cycle, the FP32 / BF16 V-cycle on
// cycle-precision vectors, and the SGS preconditioner (FP64, or FP32 vectors).
bcs_status precond_cycle64(Solver* s, const double* v, double* z);
bcs_status precond_cycle32(Solver* s, const float* v, float* z);
bcs_status sgs_fixed(Solver* s, const void* v, void* z);
bool cycle_is_float(const Solver* s);


template <class TI, class TO>
bcs_status cast_vec(Solver* s, const TI* in, TO* out, size_t N);

// ------------------------------------------------------------------- setup.cu
bcs_status amg_setup(Solver* s, bool full);
// Multicolour DILU of level L: colouring and colour lists when full, then
// the FP64 factor (E_i^{-1}); marks the level block-Jacobi (ncol = -1) when
// it would need more than 128 colours.
// sgs: E = D (multicolour block SGS) instead of the DILU factor
bcs_status dilu_setup(Solver* s, Level& L, bool full, bool sgs);
// FP32 copies of a DILU level for the FP32 / BF16 cycle.
bcs_status dilu_prepare(Solver* s, Level& L);

// ------------------------------------------------------------------ krylov.cu
bcs_status solve(Solver* s, const double* b_d, double* x_d, bcs_result* res);
// FGMRES of count solvers in lockstep (device arrays b[i], x[i]; all work on
// ss[0]'s stream); res[i] per solver.
bcs_status solve_batch(Solver* const* ss, int count, const double* const* b, double* const* x, bcs_result* res);

}  // namespace bcs

struct bcs_solver {
  bcs::Solver impl;
};
