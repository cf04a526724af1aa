/*
 * bcs.h - block-coupled sparse solver for one B300 GPU (C ABI).
 *
 * Solves A x = b where A is the block-coupled matrix of Eq. 1 (Sec. 2):
 *     A_ii U_i + sum_{j in N(i)} A_ij U_j = b_i,
 * every A_ij a dense n x n block (n = 5 for the density-based solver of
 * Sec. 2.1, n = 4 for the pressure-based solver of Sec. 2.2; any 1 <= n <= 8
 * is accepted). The matrix arrives in OpenFOAM's LDU face form (Sec. 2.3):
 * per internal face f an owner cell owner[f] and a neighbour cell
 * neighbour[f]; upper[f] is the block at (row owner, column neighbour),
 * lower[f] the block at (row neighbour, column owner); diag[i] is A_ii. Blocks
 * are stored "block AoS" (Sec. 2.3): each block row-major, blocks
 * concatenated; vectors are cell-major, component-minor ([cell][n]).
 *
 * The calls follow the paper's per-iteration procedure (Alg. 1): create a
 * solver once; upload the face addressing on the first iteration or after a
 * topology change (bcs_set_structure); upload coefficients every iteration
 * (bcs_set_values: the first upload after a structure change runs the full
 * AMG setup, later ones replace values on the fixed sparsity); solve b -> x to
 * a relative tolerance (bcs_solve); read iterations and residuals
 * (bcs_result); destroy on the final iteration. The solver is a Krylov method
 * (FGMRES or BiCGStab, Sec. 2.3) preconditioned with aggregation AMG.
 *
 * Memory: every pointer argument is either host memory (mem = BCS_MEM_HOST)
 * or device memory of the solver's device (mem = BCS_MEM_DEVICE), as the
 * argument's comment says. The caller owns every array it passes; the library
 * copies what it keeps, so inputs may be freed once the call returns. Every
 * call below synchronises the solver's stream before returning.
 *
 * Errors: every call returns a bcs_status; no call aborts the process. The
 * message of the last failure is available from bcs_last_error(). After
 * BCS_ECUDA the solver should be destroyed.
 */
#ifndef BCS_H
#define BCS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define BCS_API __attribute__((visibility("default")))
#else
#define BCS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum bcs_status {
  BCS_OK = 0,
  BCS_EINVAL = 1,          /* invalid argument or addressing */
  BCS_ENOMEM = 2,          /* device allocation failed */
  BCS_ECUDA = 3,           /* CUDA runtime error */
  BCS_NOT_CONVERGED = 4,   /* maxiter reached above the tolerance */
  BCS_BREAKDOWN = 5,       /* NaN/Inf or a Krylov breakdown */
  BCS_SINGULAR_BLOCK = 6,  /* a diagonal block (or the coarse matrix) is singular */
  BCS_TIMEOUT = 7,         /* bcs_server_wait: the request is still running after timeout_ms */
  BCS_REJECTED = 8,        /* serving: request does not fit the memory budget */
  BCS_ESTATE = 9           /* call out of order (e.g. solve before set_values) */
} bcs_status;

enum { BCS_MEM_HOST = 0, BCS_MEM_DEVICE = 1 };
enum { BCS_FGMRES = 0, BCS_BICGSTAB = 1 };
/* BCS_PC_SGS: one application of the multicolour block symmetric
 * Gauss-Seidel (LU-SGS) preconditioner M = (D + L) D^-1 (D + U), colour
 * order as the DILU smoother (Sec. 2.1's CPU preconditioner; Sec. 5's GPU
 * GMRES + SGS runs). */
enum { BCS_PC_AMG = 0, BCS_PC_NONE = 1, BCS_PC_JACOBI = 2, BCS_PC_SGS = 3 };
enum { BCS_P_SMOOTHED = 0, BCS_P_TENTATIVE = 1 };
enum { BCS_PREC_FP64 = 0, BCS_PREC_FP32 = 1, BCS_PREC_BF16 = 2 };

/* Solver options (Alg. 1: "initialize with linear solver options"). Fill with
 * bcs_config_default(), then override fields. */
/* Smoothers of the V-cycle (Sec. 4 names DILU for the GPU runs). DILU:
 * rows are coloured (Jones-Plassmann, first-fit, lowbias32 priorities, at
 * most 128 colours; a level needing more keeps block Jacobi); j precedes i
 * when colour(j) < colour(i); E_i = A_ii - sum_{j before i} A_ij E_j^-1 A_ji;
 * M = (E + L) E^-1 (E + U); one step x <- x + M^-1 (b - A x). */
enum { BCS_SMOOTH_JACOBI = 0, BCS_SMOOTH_DILU = 1, BCS_SMOOTH_SGS = 2 };

typedef struct bcs_config {
  int solver;              /* BCS_FGMRES (default) or BCS_BICGSTAB */
  int restart;             /* FGMRES restart length m (default 30, 1..64) */
  double tol;              /* stop when ||b - A x||_2 / ||b||_2 <= tol (1e-8) */
  int maxiter;             /* Krylov iteration cap (1000) */
  int precond;             /* BCS_PC_AMG (default), BCS_PC_NONE, BCS_PC_JACOBI, BCS_PC_SGS */
  int pmode;               /* BCS_P_TENTATIVE (default) or BCS_P_SMOOTHED */
  int matching_rounds;     /* handshake rounds per matching pass (4) */
  int agg_passes;          /* matching passes per level (2: aggregates of ~4) */
  double jacobi_omega;     /* damped block-Jacobi weight (0.8) */
  int nu1, nu2;            /* pre / post smoothing sweeps (2, 2) */
  int coarse_size;         /* stop coarsening at <= this many block rows (32) */
  int max_levels;          /* hierarchy depth cap (20) */
  double max_coarsen_ratio;/* stop when C_{l+1} > ratio * C_l (0.8) */
  double p_omega;          /* smoothed P: omega_P = p_omega / rho_hat (4/3) */
  int coarse_dense_max;    /* dense inverse at the coarsest level when rows*n <= this (1024) */
  int coarse_sweeps;       /* else this many block-Jacobi sweeps there (8) */
  int precision;           /* AMG storage: BCS_PREC_FP64, BCS_PREC_FP32 (default), BCS_PREC_BF16 */
  int smoother;            /* BCS_SMOOTH_JACOBI (default, damped by jacobi_omega),
                              BCS_SMOOTH_DILU (multicolour block DILU, undamped) or
                              BCS_SMOOTH_SGS (multicolour block SGS, undamped) */
  int profile;             /* 1: time kernels with CUDA events (bcs_get_stats) */
  int profile_kinds;       /* with profile = 1: bitmask of the kernel kinds to time (bit k:
                              kind k of bcs_kernel_kind_name); 0 = every kind */
  int slice_layout;        /* FP32 / BF16 level storage: 0 one lane per scalar row, 1 one thread
                              per block row, -1 (default) timed per level at full setup and the
                              faster kept; both give identical results */
  int cycle_graph;         /* FP32 / BF16 V-cycle replayed as one CUDA graph: 0 off, 1 or -1
                              (default) on, except while profile = 1 times kernels inside
                              the cycle (per-kernel events) */
  int reorder;             /* read by bcs_set_structure: 1 = renumber the cells internally in
                              reverse Cuthill-McKee order for locality (vectors, LDU arrays and
                              results stay in the caller's numbering; bcs_get_permutation);
                              0 (default) = keep the caller's numbering */
  int tail_rows;           /* FP32 / BF16 V-cycle with block Jacobi and tentative P: the levels
                              of at most tail_rows block rows (and all coarser ones) run as one
                              thread-block-cluster launch per cycle instead of a launch per
                              sweep, residual and transfer (identical results); read at each
                              set_values; 0 (default) = off: measured on B300, the graph-replayed
                              separate launches are faster */
  int dilu_cluster_rows;   /* FP32 / BF16 cycle with the DILU or SGS smoother: on levels of at
                              most dilu_cluster_rows block rows a smoothing step (residual and
                              every colour's forward and backward sweep) runs as one launch of a
                              thread-block cluster with a cluster barrier between colours,
                              instead of 1 + 2 x colours launches (identical results); read at
                              each set_values; default 4096 (measured on B300: larger levels run
                              faster as separate full-GPU launches), 0 = off */
  int dependent_launch;    /* 1 (default): the V-cycle's kernels are launched as programmatic
                              dependent launches (each may be scheduled while the kernel before
                              it finishes, and waits for that kernel's results before touching
                              any data), which hides part of the launch gap between the many
                              short kernels of the coarse levels; 0: ordinary launches.
                              Identical results either way */
  int x0_zero;             /* 1: bcs_solve / bcs_solve_batch ignore the values x holds on entry
                              and start from x = 0 (with host memory x is then only written,
                              not copied to the device); 0 (default): x holds the initial guess */
  /* Device memory, read by bcs_create (later changes are ignored): with alloc
     and release both set, every device buffer of the solver comes from
     alloc(bytes, stream, alloc_user) and goes back through release(ptr,
     bytes, stream, alloc_user), stream being the solver's stream, on the
     thread that calls into the library; memory is used stream-ordered on that
     stream; alloc returns NULL when it cannot allocate (the call then fails
     with BCS_ENOMEM); memory must be 256-byte aligned (anything else is
     handed back and treated as a failed allocation). Both NULL (default):
     cudaMallocAsync / cudaFreeAsync on the solver's stream. Exactly one of
     them set is BCS_EINVAL. */
  void* (*alloc)(size_t bytes, void* stream, void* alloc_user);
  void (*release)(void* ptr, size_t bytes, void* stream, void* alloc_user);
  void* alloc_user;
} bcs_config;

typedef struct bcs_result {
  int status;              /* bcs_status of the solve */
  int iters;               /* Krylov iterations (BiCGStab: one per two V-cycles) */
  int restarts;            /* FGMRES restarts / BiCGStab restarts */
  int levels;              /* AMG levels */
  double rel_res_initial;  /* ||b - A x0|| / ||b|| */
  double rel_res_final;    /* true residual ||b - A x|| / ||b|| recomputed in FP64 */
  double setup_ms;         /* last set_values (conversion + AMG setup), wall time */
  double solve_ms;         /* this solve, wall time */
  int host_syncs;          /* times the host waited for the device during this solve */
} bcs_result;

/* Per-kernel-kind statistics since creation or the last bcs_reset_stats. */
#define BCS_NUM_KERNEL_KINDS 16
typedef struct bcs_stats {
  long long launches;                         /* kernels launched by this solver */
  long long kind_launches[BCS_NUM_KERNEL_KINDS];
  double kind_ms[BCS_NUM_KERNEL_KINDS];       /* CUDA-event time (profile = 1 only) */
  double kind_bytes[BCS_NUM_KERNEL_KINDS];    /* algorithmic bytes moved */
  double kind_flops[BCS_NUM_KERNEL_KINDS];    /* algorithmic flops */
} bcs_stats;

typedef struct bcs_solver bcs_solver;

/* Fill cfg with defaults. Returns BCS_EINVAL when cfg is NULL. */
BCS_API bcs_status bcs_config_default(bcs_config* cfg);

/* Create a solver for n x n blocks (1 <= n <= 8) on the current CUDA device.
 * stream: a cudaStream_t the solver launches on (NULL = legacy default
 * stream). cfg may be NULL (defaults). *out receives the handle.
 * BCS_EINVAL for a bad n or an option out of range. */
BCS_API bcs_status bcs_create(bcs_solver** out, int n, const bcs_config* cfg, void* stream);

/* Destroy the solver and free its device memory. NULL is accepted. */
BCS_API bcs_status bcs_destroy(bcs_solver* s);

/* Replace the options. A change of any AMG field (or the precision) drops the
 * hierarchy, so the next set_values runs a full setup. */
BCS_API bcs_status bcs_set_config(bcs_solver* s, const bcs_config* cfg);

/* Upload the LDU face addressing (Alg. 1, first iteration / topology change):
 * n_cells C >= 1, n_faces F >= 0, owner[F] and neighbour[F] int32 cell ids
 * (host or device per mem). Builds the block-CSR structure on the device:
 * per row the diagonal plus one block per face, columns ascending.
 * owner > neighbour is accepted (upper is still the (owner, neighbour) block).
 * BCS_EINVAL: C < 1, F < 0, an id out of range, owner == neighbour, or a
 * repeated face (unordered pair); the solver then has no structure. Drops any
 * AMG hierarchy and values. */
BCS_API bcs_status bcs_set_structure(bcs_solver* s, int32_t n_cells, int32_t n_faces,
                             const int32_t* owner, const int32_t* neighbour, int mem);

/* Upload coefficients (Alg. 1, every iteration): diag[C][n][n],
 * upper[F][n][n] (block (owner, neighbour)), lower[F][n][n] (block
 * (neighbour, owner)), FP64 row-major, host or device per mem. Permutes them
 * into block-CSR order (Alg. 1, LDU -> block CSR) and then runs the full AMG
 * setup if no hierarchy exists, else a values-only resetup that keeps the
 * aggregates and every sparsity pattern. BCS_ESTATE before set_structure;
 * BCS_SINGULAR_BLOCK when a diagonal block or the coarsest matrix is
 * singular (the hierarchy is then dropped). */
BCS_API bcs_status bcs_set_values(bcs_solver* s, const double* diag, const double* upper,
                          const double* lower, int mem);

/* Flow parameters of the density-based assembly (bcs_assemble_density). */
typedef struct bcs_flow_params {
  double gamma;    /* ratio of specific heats, > 1 (default 1.4) */
  double mu;       /* dynamic viscosity, >= 0 (default 1e-3) */
  double prandtl;  /* Prandtl number, > 0 (default 0.72) */
  double cfl;      /* pseudo-time CFL number, > 0 (default 10) */
} bcs_flow_params;

/* Fill p with the defaults above; BCS_EINVAL for NULL. */
BCS_API bcs_status bcs_flow_params_default(bcs_flow_params* p);

/* Assemble the density-based coupled system on the device (Sec. 2.1,
 * Eqs. approxJac1 / approxJac2 with the pseudo-time term of
 * Eq. discretBackward) on the structure of bcs_set_structure; n must be 5.
 * Inputs (host or device per mem): Q[C][5] = (rho, rho u, rho v, rho w,
 * rho E) per cell (ideal gas), area[F] face areas, normal[F][3] unit face
 * normals pointing from owner to neighbour, dist[F] owner-neighbour centre
 * distances. For face f with spectral radius lambda_f (Roe average of the two
 * states plus max(4/3, gamma) mu / (Pr rho~ dist)):
 *   A_oo += S/2 (J(Q_o, n) + lambda I),  upper[f] = S/2 (J(Q_nb, n) - lambda I),
 *   A_nn += S/2 (-J(Q_nb, n) + lambda I), lower[f] = S/2 (-J(Q_o, n) - lambda I),
 * J the inviscid normal-flux Jacobian, plus (sum_f lambda_f S_f / CFL) I on
 * every diagonal block (local pseudo-time step). With diag, upper and lower
 * all NULL the blocks are written straight into the solver's block-CSR values
 * and the call continues as bcs_set_values (full setup or values-only
 * resetup); otherwise diag[C][5][5], upper[F][5][5], lower[F][5][5] (in the
 * inputs' memory space) receive the LDU blocks and the solver is unchanged.
 * BCS_ESTATE before set_structure; BCS_EINVAL for n != 5, NULL inputs, bad
 * parameters, a state with rho <= 0 or p <= 0 (or NaN), area < 0 or
 * dist <= 0 (when writing the solver's values the solver is then left
 * without values until the next successful upload). */
BCS_API bcs_status bcs_assemble_density(bcs_solver* s, const double* Q, const double* area, const double* normal,
                                        const double* dist, const bcs_flow_params* prm, double* diag,
                                        double* upper, double* lower, int mem);

/* Segregated fields <-> block AoS (Alg. 1 steps 1, 5 and 15). The unknowns
 * come as nfields fields (1 <= nfields <= 8), field k with ncomp[k] >= 1
 * components per cell (1: scalar field, 3: vector field stored [cell][3]),
 * sum ncomp = n; the block unknown order is the fields' order with each
 * field's components in turn. Need bcs_set_structure (for C and F); every
 * array host or device per mem; BCS_EINVAL on a bad field split or NULL. */
/* out[C][n] from fields[k][C][ncomp[k]] (source term and solution, step 1). */
BCS_API bcs_status bcs_pack_vector(bcs_solver* s, int nfields, const int* ncomp, const double* const* fields,
                                   double* out, int mem);
/* fields[k][C][ncomp[k]] from in[C][n] (solution back to fields, step 15). */
BCS_API bcs_status bcs_unpack_vector(bcs_solver* s, int nfields, const int* ncomp, const double* in,
                                     double* const* fields, int mem);

/* One coupling of the coefficient matrix: LDU arrays of the sub-blocks of
 * row field a and column field b, diag[C][na][nb], upper[F][na][nb] (row
 * owner), lower[F][na][nb] (row neighbour), row-major; all three NULL for a
 * zero coupling. */
typedef struct bcs_coupling {
  const double* diag;
  const double* upper;
  const double* lower;
} bcs_coupling;

/* Coefficients in block AoS (step 5) from coupling[a * nfields + b]. With
 * diag, upper and lower all NULL the blocks go straight into the solver's
 * block-CSR values (step 5 and the LDU -> block-CSR permutation in one pass)
 * and the call continues as bcs_set_values (full setup or values-only
 * resetup); otherwise diag[C][n][n], upper[F][n][n], lower[F][n][n] (in the
 * inputs' memory space) receive the LDU blocks. A coupling with only some of
 * its three arrays given is BCS_EINVAL. */
BCS_API bcs_status bcs_pack_coefficients(bcs_solver* s, int nfields, const int* ncomp,
                                         const bcs_coupling* coupling, double* diag, double* upper,
                                         double* lower, int mem);

/* Forget the hierarchy: the next set_values runs a full setup (new
 * aggregates). */
BCS_API bcs_status bcs_invalidate_hierarchy(bcs_solver* s);

/* Solve A x = b: b[C][n] FP64; x[C][n] FP64 holds the initial guess on entry
 * and the solution on exit (both host or both device per mem). res may be
 * NULL. Returns BCS_OK when the true relative residual is <= tol,
 * BCS_NOT_CONVERGED at maxiter, BCS_BREAKDOWN on NaN/Inf or breakdown;
 * x holds the last iterate in every case. b = 0 gives x = 0 and BCS_OK.
 * BCS_ESTATE before set_values. */
BCS_API bcs_status bcs_solve(bcs_solver* s, const double* b, double* x, int mem, bcs_result* res);

/* y = A x with the fine matrix in FP64 (Eq. 1 left-hand side); x, y [C][n]
 * host or device per mem. BCS_ESTATE before set_values. */
BCS_API bcs_status bcs_spmv(bcs_solver* s, const double* x, double* y, int mem);

/* z = M^{-1} v: one application of the configured preconditioner (one AMG
 * V-cycle from zero) in the configured precision, returned in FP64. */
BCS_API bcs_status bcs_precond_apply(bcs_solver* s, const double* v, double* z, int mem);

/* perm[C] (HOST, caller-owned): the caller's cell of every internal row
 * (the identity unless the structure was built with cfg.reorder = 1, the
 * reverse Cuthill-McKee order standing in for Sec. 2.3's renumbering).
 * BCS_ESTATE before bcs_set_structure, BCS_EINVAL for NULL. */
BCS_API bcs_status bcs_get_permutation(bcs_solver* s, int32_t* perm);

/* Test hooks: copies of internal state to HOST arrays (any may be NULL).
 * bcs_get_bsr: row_ptr[C+1], col[nnz], val[nnz][n][n] of the fine matrix and
 * the LDU -> BSR maps pos_diag[C], pos_up[F], pos_lo[F]. Matrices and level
 * data are in the internal row numbering (bcs_get_permutation maps it to the
 * caller's cells when cfg.reorder = 1); pos_diag is indexed by the caller's
 * cell, pos_up / pos_lo by face. */
BCS_API bcs_status bcs_get_bsr(bcs_solver* s, int32_t* row_ptr, int32_t* col, double* val,
                       int32_t* pos_diag, int32_t* pos_up, int32_t* pos_lo);
/* Number of AMG levels (0 without a hierarchy). */
BCS_API int bcs_num_levels(const bcs_solver* s);
/* Sizes of level l: block rows, nnz blocks of A_l, nnz blocks of P_l (0 at
 * the coarsest level or in tentative mode), coarse_kind (-1 not coarsest,
 * 0 dense inverse, 1 smoother sweeps). */
BCS_API bcs_status bcs_get_level_info(const bcs_solver* s, int l, int* rows, int* nnz, int* p_nnz,
                              int* coarse_kind);
/* FP64 level data: A_l (row_ptr, col, val), aggregate map agg[rows] (not at
 * the coarsest level), block inverses dinv[rows][n][n]. */
BCS_API bcs_status bcs_get_level(bcs_solver* s, int l, int32_t* row_ptr, int32_t* col, double* val,
                         int32_t* agg, double* dinv);
/* Smoothed prolongation of level l (pmode smoothed only) and omega_P. */
BCS_API bcs_status bcs_get_prolongation(bcs_solver* s, int l, int32_t* row_ptr, int32_t* col,
                                double* val, double* omega_p);
/* Dense inverse of the coarsest matrix, [N][N] with N = rows * n. */
BCS_API bcs_status bcs_get_coarse_inverse(bcs_solver* s, double* inv);
/* DILU data of level l (smoother = BCS_SMOOTH_DILU): *ncolours = number of
 * colours, or -1 when the level keeps block Jacobi (then nothing is copied);
 * colour[rows] and einv[rows][n][n] (FP64 E_i^{-1}) may be NULL. */
BCS_API bcs_status bcs_get_dilu(bcs_solver* s, int level, int* ncolours, int32_t* colour, double* einv);

/* Statistics (launch counts always; times only with cfg.profile = 1). */
BCS_API bcs_status bcs_get_stats(bcs_solver* s, bcs_stats* st);
BCS_API bcs_status bcs_reset_stats(bcs_solver* s);
/* Per-kernel timing table (cfg.profile = 1): one line per kernel,
 * "name<TAB>launches<TAB>ms<TAB>algorithmic bytes<TAB>kind", written to buf
 * (NUL terminated); BCS_EINVAL when it does not fit in len bytes. */
BCS_API bcs_status bcs_get_kernel_times(bcs_solver* s, char* buf, size_t len);
/* Per-level totals of the timed launches (cfg.profile = 1) since the last
 * bcs_reset_stats: launches[k], ms[k] (CUDA-event time) and bytes[k]
 * (algorithmic bytes) of kernel kind k on hierarchy level `level`, for
 * k < BCS_NUM_KERNEL_KINDS (caller-owned host arrays of that length). A
 * launch belongs to the level whose matrix it reads or builds: setup work of
 * level l (its block inverses, the aggregation of its rows, the Galerkin
 * product that forms level l + 1), its FP32 / BF16 copies, and its sweeps,
 * residuals and transfers in the V-cycle. Zeros for a level with no timed
 * launch; BCS_EINVAL for level outside [0, 64). */
BCS_API bcs_status bcs_get_level_times(bcs_solver* s, int level, long long* launches, double* ms, double* bytes);
/* Name of kernel kind k (0 <= k < BCS_NUM_KERNEL_KINDS), "" if unused. */
BCS_API const char* bcs_kernel_kind_name(int k);

/* ---- Serving: continuous batching of solves from many cases ----------
 * A server owns worker threads ("slots") on the current device. A case is a
 * fixed LDU face addressing (Alg. 1: the structure set up on the first
 * iteration); each request brings one later iteration's coefficients and
 * right-hand side for a case. Requests are taken in arrival order, skipping
 * those whose case is busy or does not fit yet; a case's requests run one at a
 * time in submission order (values-only resetup of its resident hierarchy,
 * then a solve), different cases run concurrently on their own streams.
 * Cases are admitted while their device footprint fits in budget_bytes,
 * evicting least-recently-used idle cases; a case larger than the budget is
 * answered with BCS_REJECTED. Results are deterministic per case, the same
 * alone or in any mix. */
/* Largest batch of bcs_solve_batch and of a server's batching. */
#define BCS_BATCH_MAX 64

typedef struct bcs_server bcs_server;

typedef struct bcs_server_stats {
  long long submitted, completed, rejected, evictions, admissions, queued;
  size_t resident_bytes, budget_bytes;
  int resident_cases;
  double p50_ms, p99_ms, mean_ms;   /* submit -> completion latency */
  /* GPU timeline since the last reset: each request's interval runs from an
   * event recorded on its case's stream before the resetup to one recorded
   * after the solve. window_ms: first start to last end; busy_frac: share
   * of the window covered by at least one request; overlap_frac: share
   * covered by two or more (their kernels in flight together);
   * mean_in_flight: summed interval lengths over the window. */
  double window_ms, busy_frac, overlap_frac, mean_in_flight;
  long long batches, batched_requests;  /* batched solves run and the requests they served */
} bcs_server_stats;

/* budget_bytes = 0: 80 % of the device's free memory. slots: 1..64. cfg may
 * be NULL (defaults). */
BCS_API bcs_status bcs_server_create(bcs_server** out, size_t budget_bytes, int slots, const bcs_config* cfg);
/* Finishes every queued request, then frees everything. */
BCS_API bcs_status bcs_server_destroy(bcs_server* srv);
/* Copies the face addressing (HOST arrays) of a case with n x n blocks. */
BCS_API bcs_status bcs_server_register_case(bcs_server* srv, int n, int32_t n_cells, int32_t n_faces,
                                            const int32_t* owner, const int32_t* neighbour, int* case_id);
/* Queue a solve: arrays diag[C][n][n], upper / lower[F][n][n], b[C][n];
 * x[C][n] holds the initial guess and receives the solution. mem says where
 * all five live: BCS_MEM_HOST, or BCS_MEM_DEVICE (memory of the device the
 * server was created on, complete before this call: the request runs on the
 * case's own stream). The arrays must stay valid until the request
 * completes. */
BCS_API bcs_status bcs_server_submit(bcs_server* srv, int case_id, const double* diag, const double* upper,
                                    const double* lower, const double* b, double* x, int mem, int64_t* ticket);
/* Wait for a request (timeout_ms < 0: no limit); returns the request's
 * status (BCS_TIMEOUT when still running after timeout_ms, the ticket then
 * stays valid). res and latency_ms (submit -> completion) may be NULL. */
BCS_API bcs_status bcs_server_wait(bcs_server* srv, int64_t ticket, int timeout_ms, bcs_result* res,
                                  double* latency_ms);
/* Batching (default 1: off): a slot that takes a request of a resident case
 * also takes the first queued request of up to max_batch - 1 other idle
 * resident cases with the same block size and memory kind, runs each
 * case's values-only resetup and solves them together with
 * bcs_solve_batch (each result equal to the case's solve alone; a batch the
 * batched solver refuses is solved case by case). 1 <= max_batch <=
 * BCS_BATCH_MAX, else BCS_EINVAL. */
BCS_API bcs_status bcs_server_set_batch(bcs_server* srv, int max_batch);
BCS_API bcs_status bcs_server_get_stats(bcs_server* srv, bcs_server_stats* st);
BCS_API bcs_status bcs_server_reset_stats(bcs_server* srv);
/* The message of the most recent request that failed with BCS_ECUDA,
 * BCS_ENOMEM, BCS_SINGULAR_BLOCK or BCS_EINVAL (the case's device state is
 * dropped after such a failure, its solver's message with it), NUL
 * terminated and truncated to len bytes; "" when none failed. */
BCS_API bcs_status bcs_server_last_error(bcs_server* srv, char* buf, size_t len);

/* Allocation-free block-CSR structure build (the paper has no counterpart).
 * For callers that cannot let a library allocate device memory: programs that
 * reserve the GPU's memory up front under a hard budget, and programs that
 * forbid cudaMalloc / cudaFree after start-up because those calls synchronise
 * the device and stall their other streams. Builds exactly what
 * bcs_set_structure builds (row_ptr[C+1], col[C+2F], pos_diag[C], pos_up[F],
 * pos_lo[F], all int32 DEVICE arrays owned by the caller) from DEVICE arrays
 * owner[F], neighbour[F], launching on `stream` (a cudaStream_t, NULL = legacy
 * default stream) and synchronising it before returning. It allocates
 * nothing: its scratch lives in a fixed ~4 MB device array inside the library
 * that every GPU loading the library keeps until the process exits. Limit:
 * n_cells <= 1048576; larger sizes return BCS_EINVAL with a message. Before
 * any launch every array is checked to be device memory of the current
 * device (cudaPointerGetAttributes); a host pointer returns BCS_EINVAL with
 * nothing launched. The call reads one status word back from the device
 * once, at the end, and waits for the stream there. The first call on each
 * device, with that device current, looks up the fixed array's device
 * address and keeps it for the process (make that first call before any
 * stream capture); the kept address does not survive a reset of the
 * device's primary context (cudaDeviceReset), so do not call this entry
 * point after one. All calls share the scratch and it keeps the last call's
 * contents (the kernels clear what must start at zero), so calls that
 * overlap on the GPU race; serialise them. Errors as bcs_set_structure
 * (bad cell ids, owner == neighbour, a repeated face); when err is not NULL,
 * a message of at most errlen bytes is written there. */
BCS_API bcs_status bcs_ldu_structure_noalloc(int32_t n_cells, int32_t n_faces, const int32_t* owner,
                                             const int32_t* neighbour, int32_t* row_ptr, int32_t* col,
                                             int32_t* pos_diag, int32_t* pos_up, int32_t* pos_lo,
                                             void* stream, char* err, size_t errlen);

/* Solve `count` systems together (1 <= count <= BCS_BATCH_MAX): solvers[i]
 * with b[i][C_i][n] and x[i][C_i][n] (x[i] holds x0 on entry, the solution on
 * return), all arrays in `mem` (BCS_MEM_HOST or BCS_MEM_DEVICE). The systems
 * may differ in size and hierarchy depth; their FGMRES iterations run in
 * lockstep, every step's kernels covering all systems at once (one launch
 * per V-cycle phase and level for the whole batch), each system stopping on
 * its own test. Every system's iterates, x and result equal those of
 * bcs_solve on it alone, bit for bit. The paper has no counterpart (its
 * linear systems are solved one by one); batching serves many small
 * independent cases. Requires, for every solver: values set (else
 * BCS_ESTATE), the same block size, FGMRES, an FP32 or BF16 aggregation-AMG
 * cycle with block Jacobi and tentative prolongation, the same nu1, nu2,
 * jacobi_omega, coarse_sweeps and restart, no internal renumbering, all on
 * the current device (else BCS_EINVAL, message on solvers[0]). The work runs
 * on solvers[0]'s stream after every solver's stream is synchronised; the
 * call returns when it is complete. res[i] receives system i's result; the
 * return value is BCS_OK, or the first non-OK status among the systems. */
BCS_API bcs_status bcs_solve_batch(bcs_solver* const* solvers, int count, const double* const* b, double* const* x,
                                   int mem, bcs_result* res);

/* Message for the last failed call on s (never NULL). */
BCS_API const char* bcs_last_error(const bcs_solver* s);

/* Device bytes currently held by the solver. */
BCS_API size_t bcs_device_bytes(const bcs_solver* s);

#ifdef __cplusplus
}
#endif
#endif /* BCS_H */
