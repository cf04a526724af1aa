/*
 * FP64 CPU oracle for the block-coupled linear solve.
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, single-threaded reference
 * written from the paper's statement of the problem; it shares no code with
 * the CUDA library. Only the tests, the package's smoke() check and the
 * benchmark's CPU-baseline leg may load it. The product path never calls it.
 *
 * What it follows:
 *   Eq. 1 (Sec. 2)        A_ii U_i + sum_N A_ij U_j = b_i with dense n x n
 *                         blocks; LDU face addressing (Sec. 2.3): upper[f] is
 *                         the block at (owner, neighbour), lower[f] the block
 *                         at (neighbour, owner).
 *   Sec. 2.3, Alg. 1      block AoS storage (row-major n x n blocks,
 *                         concatenated) and the LDU -> block-CSR permutation;
 *                         first-iteration setup vs. values-only replacement.
 *   Sec. 2.3              aggregation AMG for block systems built by graph
 *                         matching, smoothers, Krylov solvers (GMRES, BiCGStab).
 *   Sec. 2 (ref. Saad & Schultz)  GMRES.
 *   Sec. 2.1, Eqs. approxJac1/2   assembly of the density-based blocks from
 *                         cell states and face geometry (assembly.cpp).
 *   Sec. 2.1 / Sec. 5     LU-SGS / SGS preconditioning (multicolour block SGS,
 *                         precond = 3, smoother = 2).
 *   Sec. 2.3              cell renumbering: reverse Cuthill-McKee
 *                         (reorder.cpp). The segregated-field <-> block AoS
 *                         conversions of Alg. 1 steps 1, 5, 15 are plain numpy
 *                         definitions in __init__.py.
 * The paper leaves the AMG and Krylov details unspecified; the readings used
 * here (matching rule, smoothed prolongation, block-Jacobi smoother, CGS2,
 * stopping rule, coarse solve) are written out beside each function.
 *
 * Parity status: every function below is pinned by the CPU tests against
 * closed forms, invariants, dense/library special cases or brute force, except
 * where a header comment says "parity unpinned".
 */
#ifndef BCS_ORACLE_H
#define BCS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Solver settings read by the oracle. Field meaning matches the library's
 * configuration; the two structs are deliberately separate definitions. */
typedef struct {
  int solver;            /* 0 = FGMRES(restart), 1 = BiCGStab */
  int restart;           /* FGMRES restart length m */
  double tol;            /* relative residual target ||b - A x|| / ||b|| */
  int maxiter;           /* total Krylov iterations allowed */
  int precond;           /* 0 = AMG V-cycle, 1 = none, 2 = block Jacobi (one sweep),
                            3 = multicolour block SGS (one application of M^-1) */
  int pmode;             /* 0 = smoothed prolongation, 1 = tentative (default) */
  int matching_rounds;   /* synchronous handshake rounds per matching pass */
  int agg_passes;        /* matching passes per level (2 gives aggregates of ~4) */
  double jacobi_omega;   /* damped block-Jacobi weight */
  int nu1, nu2;          /* pre / post smoothing sweeps */
  int coarse_size;       /* stop coarsening when rows <= coarse_size */
  int max_levels;        /* hierarchy depth limit */
  double max_coarsen_ratio; /* stop if C_{l+1} > ratio * C_l */
  double p_omega;        /* prolongation smoothing numerator: omega_P = p_omega / rho */
  int coarse_dense_max;  /* dense inverse at the coarsest level if rows*n <= this */
  int coarse_sweeps;     /* otherwise this many smoother sweeps */
  int smoother;          /* 0 = damped block Jacobi, 1 = multicolour block DILU,
                            2 = multicolour block SGS */
} or_config;

typedef struct {
  int status;            /* 0 ok, 4 not converged, 5 breakdown, 6 singular block */
  int iters;
  int restarts;
  double rel_res_initial;
  double rel_res_final;  /* true residual, recomputed */
  int levels;
} or_result;

void or_config_default(or_config* cfg);

/* LDU addressing check: returns 0 when valid; 1 when C < 1, F < 0, an index is
 * out of range, owner == neighbour, or a face (as an unordered pair) repeats. */
int or_ldu_check(int C, int F, const int32_t* owner, const int32_t* neighbour);

/* Block-CSR structure of the LDU matrix (Sec. 2.3). Rows hold the diagonal and
 * one block per face touching the row, columns strictly ascending.
 * row_ptr[C+1], col[C+2F], pos_diag[C], pos_up[F], pos_lo[F]. Returns the
 * result of or_ldu_check. */
int or_ldu_structure(int C, int F, const int32_t* owner, const int32_t* neighbour,
                     int32_t* row_ptr, int32_t* col, int32_t* pos_diag,
                     int32_t* pos_up, int32_t* pos_lo);

/* BSR values from LDU block arrays (Alg. 1, LDU -> block CSR permutation). */
void or_ldu_values(int C, int F, int n, const int32_t* pos_diag, const int32_t* pos_up,
                   const int32_t* pos_lo, const double* diag, const double* upper,
                   const double* lower, double* val);

/* Inverse of or_ldu_values: BSR values back to LDU block arrays. */
void or_bsr_to_ldu(int C, int F, int n, const int32_t* pos_diag, const int32_t* pos_up,
                   const int32_t* pos_lo, const double* val, double* diag, double* upper,
                   double* lower);

/* y = A x for a BSR matrix with `rows` block rows (Eq. 1 left-hand side). */
void or_bsr_spmv(int rows, int n, const int32_t* row_ptr, const int32_t* col,
                 const double* val, const double* x, double* y);

/* Gauss-Jordan inverse with implicit partial pivoting of an N x N row-major
 * matrix. Returns 0, or 1 when a pivot is exactly zero. */
int or_dense_inverse(int N, const double* A, double* Ainv);

/* Frobenius norm of each n x n block (fma accumulation, row-major order). */
void or_block_norms(int nblocks, int n, const double* val, double* nrm);

/* One aggregation level: matching passes + leftovers + canonical numbering.
 * agg[rows] receives aggregate ids; returns the number of aggregates. */
int or_aggregate(int rows, int n, const int32_t* row_ptr, const int32_t* col,
                 const double* val, const or_config* cfg, int32_t* agg);

/* ---- multicolour block DILU (Sec. 4: the GPU runs' smoother) ---------- *
 * Colouring: synchronous Jones-Plassmann rounds. Row priority = (h(i), i)
 * with h the 32-bit "lowbias32" integer hash (xorshift-multiply, constants
 * 0x7feb352d and 0x846ca68b). In a round every uncoloured row whose priority
 * exceeds that of all its uncoloured neighbours takes the smallest colour
 * not held by a neighbour coloured in an earlier round. Returns the number
 * of colours, or -1 if some row would need colour >= 128 (the level then
 * keeps block Jacobi). colour[rows].
 * Factor (j before i iff colour(j) < colour(i)):
 *   E_i = A_ii - sum over j before i, A_ij != 0, columns ascending, of
 *         (A_ij E_j^{-1}) A_ji, each block product an fma chain from +0;
 *   einv_i = E_i^{-1} (Gauss-Jordan as or_dense_inverse). Returns 0 or 1
 *   (singular E_i).
 * Apply z = M^{-1} r, M = (E + L) E^{-1} (E + U), L / U the blocks A_ij with
 * j before / after i: forward y_i = E_i^{-1} (r_i - sum_{j before i} A_ij y_j)
 * by colours ascending, backward z_i = y_i - E_i^{-1} sum_{j after i} A_ij z_j
 * by colours descending. The smoother step is x <- x + M^{-1} (b - A x). */
int or_colour(int rows, const int32_t* row_ptr, const int32_t* col, int32_t* colour);
int or_dilu_factor(int rows, int n, const int32_t* row_ptr, const int32_t* col, const double* val,
                   const int32_t* colour, double* einv);
void or_dilu_apply(int rows, int n, const int32_t* row_ptr, const int32_t* col, const double* val,
                   const int32_t* colour, int ncolours, const double* einv, const double* r, double* z);

/* ---- AMG hierarchy ---------------------------------------------------- */
typedef struct or_amg or_amg;

/* Full setup from a fine BSR matrix (values copied). *status: 0 ok,
 * 6 singular block. */
or_amg* or_amg_setup(int rows, int n, const int32_t* row_ptr, const int32_t* col,
                     const double* val, const or_config* cfg, int* status);
/* Values-only resetup: same aggregates and sparsity, new fine values. */
int or_amg_resetup(or_amg* h, const double* val);
void or_amg_free(or_amg* h);
int or_amg_levels(const or_amg* h);
/* Sizes of level l: block rows, nnz blocks of A_l, nnz blocks of P_l (0 at
 * the coarsest level), coarse_kind (0 dense inverse, 1 smoother sweeps,
 * -1 not the coarsest). */
void or_amg_level_info(const or_amg* h, int l, int* rows, int* nnz, int* p_nnz,
                       int* coarse_kind);
/* Copies of level-l data; any pointer may be NULL. */
void or_amg_get_A(const or_amg* h, int l, int32_t* row_ptr, int32_t* col, double* val);
void or_amg_get_P(const or_amg* h, int l, int32_t* row_ptr, int32_t* col, double* val,
                  int32_t* agg, double* omega_p);
void or_amg_get_dinv(const or_amg* h, int l, double* dinv);
/* DILU data of level l (smoother = 1): returns the number of colours (-1 when
 * the level keeps block Jacobi); colour[rows] and einv[rows][n][n] may be NULL. */
int or_amg_get_dilu(const or_amg* h, int l, int32_t* colour, double* einv);
void or_amg_get_coarse_inverse(const or_amg* h, double* inv);
/* z = M^{-1} v: one V-cycle from a zero initial guess. */
void or_amg_vcycle(const or_amg* h, const double* v, double* z);

/* Solve A x = b (x holds x0 on entry). h may be NULL when cfg->precond != 0. */
int or_solve(int rows, int n, const int32_t* row_ptr, const int32_t* col,
             const double* val, const or_amg* h, const or_config* cfg,
             const double* b, double* x, or_result* res, double* hist, int hist_len);

/* As or_solve; BiCGStab (solver = 1) also records, for each of the first
 * trace_len iterations, its iterate x_k in xtrace[k][rows*n] and the
 * residual its recurrence carries for x_k in rtrace[k][rows*n] (r_k after a
 * full step, s after a half step that ends the solve). Returns the number of
 * iterations recorded (the status when nothing is traced). Test hook. */
int or_solve_trace(int rows, int n, const int32_t* row_ptr, const int32_t* col,
                   const double* val, const or_amg* h, const or_config* cfg,
                   const double* b, double* x, or_result* res, double* hist, int hist_len,
                   double* xtrace, double* rtrace, int trace_len);

/* Arnoldi check hook: runs j_steps of FGMRES's Arnoldi process from x0 = 0 and
 * returns V (j+1 vectors) and Z (j vectors), H ((j+1) x j, row-major). */
int or_fgmres_arnoldi(int rows, int n, const int32_t* row_ptr, const int32_t* col,
                      const double* val, const or_amg* h, const or_config* cfg,
                      const double* b, int j_steps, double* V, double* Z, double* H);

/* ---- Assembly of the density-based system (assembly.cpp) -------------- */
/* Sec. 2.1, Eqs. approxJac1 / approxJac2 and Eq. discretBackward. Q per cell
 * = (rho, rho u, rho v, rho w, rho E), ideal gas with ratio gamma. Returns 0,
 * or 1 for an invalid state (rho <= 0 or p <= 0) or parameter. */
int or_euler_flux(const double* Q, const double* n, double gamma, double* F);
int or_flux_jacobian(const double* Q, const double* n, double gamma, double* J);
int or_face_lambda(const double* Qo, const double* Qn, const double* n, double d, double gamma, double mu,
                   double prandtl, double* lam);
/* diag[C][5][5], upper / lower[F][5][5] of the LDU input (upper = block
 * (owner, neighbour)); normal[F][3] unit, from owner to neighbour. */
int or_assemble_density(int C, int F, const int32_t* owner, const int32_t* nb, const double* Q,
                        const double* area, const double* normal, const double* dist, double gamma, double mu,
                        double prandtl, double cfl, double* diag, double* upper, double* lower);

/* ---- Locality ordering (reorder.cpp) ---------------------------------- */
/* Reverse Cuthill-McKee order of the cell graph (one edge per face):
 * perm[new] = old. Returns 0, or 1 for a bad face. */
int or_rcm(int C, int F, const int32_t* owner, const int32_t* nb, int32_t* perm);

#ifdef __cplusplus
}
#endif
#endif
