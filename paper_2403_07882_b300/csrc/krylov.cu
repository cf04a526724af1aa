// Krylov solvers (Sec. 2.3: GMRES and BiCGStab with an AMG preconditioner).
//
// FGMRES(m): right-preconditioned flexible GMRES (GMRES of Saad & Schultz;
// flexible because the mixed-precision preconditioner is not a fixed linear
// operator), classical Gram-Schmidt applied twice, Givens rotations, restart
// after m steps. With the AMG or SGS preconditioner and graphs enabled, each
// restart cycle runs on the device (see fgmres below); otherwise the Givens
// rotations run on the host after one scalar read per step. A cycle ends
// when the rotated residual |g_{j+1}| <= tol ||b||; convergence is decided on the true residual
// ||b - A x|| / ||b|| recomputed in FP64 at every cycle end. Happy breakdown
// when h_{j+1,j} <= 1e-14 ||A z_j||.
//
// BiCGStab (van der Vorst), right-preconditioned, r_hat = r_0; a converged
// recurrence residual is confirmed with the true residual and the iteration
// restarted from it otherwise; rho = 0, (r_hat, v) = 0 or (t, t) = 0 restart
// once from the true residual, a second time report breakdown.
//
// All vectors are FP64 on the device; the preconditioner output z is stored
// in the cycle precision (FP32 in mixed mode, exactly representable in FP64).
#include <chrono>
#include <cmath>

#include "internal.h"

namespace bcs {

namespace {


size_t zbytes(const Solver* s) { return cycle_is_float(s) ? sizeof(float) : sizeof(double); }

// z = M^{-1} v (z in the cycle precision)
bcs_status apply_M(Solver* s, const double* v, void* z, size_t N) {
  switch (s->setup_cfg.precond) {
    case BCS_PC_AMG:
      return precond_apply(s, v, z);
    case BCS_PC_JACOBI:
      return jacobi_apply(s, v, (double*)z);
    case BCS_PC_SGS:
      return sgs_apply(s, v, z);
    default:
      BCS_CU(s, cudaMemcpyAsync(z, v, N * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
      return BCS_OK;
  }
}

// y = A z for a preconditioned vector z in the cycle precision. An FP32 z is
// widened once into s->kt first: converting inside the SpMV would cost one
// F32->F64 conversion per matrix entry on the FP64 pipe, as many as the FMAs.
bcs_status apply_A(Solver* s, const void* z, double* y, size_t N) {
  const void* x = z;
  if (cycle_is_float(s)) {
    BCS_ALLOC(s, s->kt, N);
    BCS_OKR(cast_vec<float, double>(s, (const float*)z, s->kt.p, N));
    x = s->kt.p;
  }
  return spmv64(s, s->lv[0].A, x, false, y, nullptr, K_SPMV64);
}

bcs_status norm(Solver* s, const double* x, size_t N, double* out) {
  BCS_OKR(dot(s, x, x, N, SLOT_N));
  BCS_OKR(fetch_scalars(s, SLOT_N + 1));
  *out = std::sqrt(s->hscal[SLOT_N]);
  return BCS_OK;
}

// r = b - A x, returns ||r||
bcs_status true_residual(Solver* s, const double* b, const double* x, double* r, size_t N, double* rn) {
  BCS_OKR(spmv64(s, s->lv[0].A, x, false, r, b, K_SPMV64));
  return norm(s, r, N, rn);
}

// ||b|| and the initial residual r = b - A x, ||r||. When x is exactly zero
// the product is skipped: b - A 0 = b element by element, so r is a copy of b
// and ||r|| = ||b|| (the same reduction over the same values).
bcs_status initial_residual(Solver* s, const double* b, const double* x, double* r, size_t N, double* bnorm,
                            double* rnorm) {
  BCS_OKR(dot(s, b, b, N, SLOT_N));
  BCS_OKR(any_nonzero(s, x, N, SLOT_X));
  BCS_OKR(fetch_scalars(s, SLOT_X + 1));
  *bnorm = std::sqrt(s->hscal[SLOT_N]);
  if (s->hscal[SLOT_X] != 0.0) return true_residual(s, b, x, r, N, rnorm);
  BCS_CU(s, cudaMemcpyAsync(r, b, N * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
  *rnorm = *bnorm;
  return BCS_OK;
}

// ---- device-resident restart cycle ------------------------------------------
// One FGMRES restart cycle without host round trips: the Arnoldi step (the
// preconditioner on fixed buffers, the outer SpMV into s->kw, both CGS2
// passes, the Givens update and stop test of k_ks_givens, v_{j+1}) is
// captured once into the body of a CUDA graph WHILE node, whose condition the
// Givens kernel clears when the cycle ends (convergence estimate, happy
// breakdown, breakdown, iteration limit, or m steps). The host then sees one
// status read per restart cycle (with the true residual) instead of one per
// iteration. The step index lives in KrylovState, so every replay of the body
// is the same graph.

// Kinds launched inside the captured step: per-kernel events there would need
// event nodes, which a conditional body cannot hold.
constexpr int LOOP_KINDS = (1 << K_SPMV64) | (1 << K_SWEEP) | (1 << K_RESID) | (1 << K_TRANSFER) | (1 << K_COARSE) |
                           (1 << K_BLAS) | (1 << K_CAST);

bool device_cycle_ok(const Solver* s) {
  if (s->cfg.cycle_graph == 0) return false;
  const int pc = s->setup_cfg.precond;
  if (pc != BCS_PC_AMG && pc != BCS_PC_SGS) return false;
  if (pc == BCS_PC_AMG && s->lv.empty()) return false;
  if (s->cfg.profile && (s->cfg.profile_kinds == 0 || (s->cfg.profile_kinds & LOOP_KINDS))) return false;
  return s->cfg.restart <= KS_MAXM;
}

// The preconditioner from its fixed input (lv[0].vb in the cycle precision,
// or s->kvj in FP64) to its fixed output (lv[0].vx, or s->kzj).
bcs_status apply_M_fixed(Solver* s) {
  Level& L0 = s->lv[0];
  const int pc = s->setup_cfg.precond, prec = s->setup_cfg.precision;
  if (prec == BCS_PREC_FP64) {
    if (pc == BCS_PC_AMG) return precond_cycle64(s, s->kvj.p, s->kzj.p);
    return sgs_fixed(s, s->kvj.p, s->kzj.p);
  }
  if (pc == BCS_PC_AMG) return precond_cycle32(s, (const float*)L0.vb.p, (float*)L0.vx.p);
  return sgs_fixed(s, L0.vb.p, L0.vx.p);
}

// One Arnoldi step of the device-resident cycle (the body of the WHILE node).
bcs_status arnoldi_step_dev(Solver* s, KrylovState* ks, cudaGraphConditionalHandle cond) {
  const size_t N = (size_t)s->C * s->n;
  const bool zf = cycle_is_float(s);
  double* V = s->kv.p;
  double* w = s->kw.p;
  BCS_OKR(ks_take_vj(s, V, N, ks, zf ? (void*)s->lv[0].vb.p : (void*)s->kvj.p, zf, N));
  BCS_OKR(apply_M_fixed(s));
  BCS_OKR(ks_store_z(s, zf ? (const void*)s->lv[0].vx.p : (const void*)s->kzj.p, zf, s->kz.p, ks,
                     zf ? s->kt.p : nullptr, N));
  BCS_OKR(spmv64(s, s->lv[0].A, zf ? (const void*)s->kt.p : (const void*)s->kzj.p, false, w, nullptr, K_SPMV64));
  BCS_OKR(ks_multidot(s, V, N, ks, w, true, N, SLOT_A));
  BCS_OKR(ks_gs_update(s, V, N, ks, s->scal.p + SLOT_A, w, N, -1));
  BCS_OKR(ks_multidot(s, V, N, ks, w, false, N, SLOT_B));
  BCS_OKR(ks_gs_update(s, V, N, ks, s->scal.p + SLOT_B, w, N, SLOT_N));
  BCS_OKR(ks_givens(s, ks, SLOT_A, SLOT_B, SLOT_N, cond));
  return ks_scale_next(s, ks, w, V, N, N);
}

// Builds (once per set of buffers) the executable graph: a WHILE node whose
// body is one captured Arnoldi step. Its launches are counted per executed
// step (kry_kind_*).
bcs_status capture_cycle(Solver* s, KrylovState* ks) {
  long long kl[BCS_NUM_KERNEL_KINDS];
  double kb[BCS_NUM_KERNEL_KINDS], kf[BCS_NUM_KERNEL_KINDS];
  const long long l0 = s->launches;
  for (int k = 0; k < BCS_NUM_KERNEL_KINDS; ++k) {
    kl[k] = s->kind_launches[k];
    kb[k] = s->kind_bytes[k];
    kf[k] = s->kind_flops[k];
  }
  if (!s->gstream) BCS_CU(s, cudaStreamCreateWithFlags(&s->gstream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  BCS_CU(s, cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle cond = 0;
  cudaGraphNode_t node = nullptr;
  cudaGraphNodeParams prm{};
  cudaError_t e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = cond;
    prm.conditional.type = cudaGraphCondTypeWhile;
    prm.conditional.size = 1;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &prm);
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return s->fail(BCS_ECUDA, std::string("conditional graph node: ") + cudaGetErrorString(e));
  }
  cudaGraph_t body = prm.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(s->gstream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return s->fail(BCS_ECUDA, std::string("capture into the loop body: ") + cudaGetErrorString(e));
  }
  const cudaStream_t own = s->stream;
  s->stream = s->gstream;
  const bcs_status st = arnoldi_step_dev(s, ks, cond);
  s->stream = own;
  cudaGraph_t captured = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(s->gstream, &captured);
  s->launches = l0;
  for (int k = 0; k < BCS_NUM_KERNEL_KINDS; ++k) {
    s->kry_kind_launches[k] = s->kind_launches[k] - kl[k];
    s->kry_kind_bytes[k] = s->kind_bytes[k] - kb[k];
    s->kry_kind_flops[k] = s->kind_flops[k] - kf[k];
    s->kind_launches[k] = kl[k];
    s->kind_bytes[k] = kb[k];
    s->kind_flops[k] = kf[k];
  }
  if (st != BCS_OK || ce != cudaSuccess) {
    cudaGraphDestroy(g);
    if (st != BCS_OK) return st;
    return s->fail(BCS_ECUDA, std::string("loop body capture: ") + cudaGetErrorString(ce));
  }
  const cudaError_t ie = cudaGraphInstantiate(&s->kry_exec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    s->kry_exec = nullptr;
    return s->fail(BCS_ECUDA, std::string("loop graph instantiate: ") + cudaGetErrorString(ie));
  }
  return BCS_OK;
}

// The launches of `steps` executed loop bodies, added to the statistics.
void count_steps(Solver* s, int steps) {
  for (int k = 0; k < BCS_NUM_KERNEL_KINDS; ++k) {
    s->launches += s->kry_kind_launches[k] * steps;
    s->kind_launches[k] += s->kry_kind_launches[k] * steps;
    s->kind_bytes[k] += s->kry_kind_bytes[k] * steps;
    s->kind_flops[k] += s->kry_kind_flops[k] * steps;
  }
}

bcs_status fgmres(Solver* s, const double* b, double* x, bcs_result* res) {
  const bcs_config& cfg = s->cfg;
  const int m = cfg.restart;
  const size_t N = (size_t)s->C * s->n;
  const bool zf = cycle_is_float(s);
  const bool dev = device_cycle_ok(s);
  BCS_ALLOC(s, s->kv, (size_t)(m + 1) * N);
  BCS_ALLOC(s, s->kz, (size_t)m * N * zbytes(s));
  BCS_ALLOC(s, s->kr, N);
  if (dev) {
    // everything the captured step touches exists before the capture
    BCS_ALLOC(s, s->kw, N);
    BCS_ALLOC(s, s->kst, sizeof(KrylovState));
    BCS_ALLOC(s, s->red, (size_t)72 * 1184);
    if (zf) BCS_ALLOC(s, s->kt, N);
    else {
      BCS_ALLOC(s, s->kvj, N);
      BCS_ALLOC(s, s->kzj, N);
    }
    if (s->kry_exec && (s->kry_key[0] != (const void*)s->kv.p || s->kry_key[1] != (const void*)s->kz.p ||
                        s->kry_key[2] != (const void*)s->kw.p || s->kry_key[3] != (const void*)s->kt.p ||
                        s->kry_key[4] != (const void*)s->kvj.p || s->kry_m != m)) {
      cudaGraphExecDestroy(s->kry_exec);
      s->kry_exec = nullptr;
    }
  }
  double* V = s->kv.p;
  char* Z = s->kz.p;
  double* r = s->kr.p;
  double bnorm = 0.0, beta = 0.0;
  BCS_OKR(initial_residual(s, b, x, r, N, &bnorm, &beta));
  res->iters = 0;
  res->restarts = 0;
  if (bnorm == 0.0) {
    BCS_CU(s, cudaMemsetAsync(x, 0, N * sizeof(double), s->stream));
    res->rel_res_initial = res->rel_res_final = 0.0;
    return BCS_OK;
  }
  res->rel_res_initial = res->rel_res_final = beta / bnorm;
  if (!std::isfinite(beta)) return BCS_BREAKDOWN;
  if (beta <= cfg.tol * bnorm) return BCS_OK;
  std::vector<double> H((size_t)(m + 1) * m, 0.0), g(m + 1), cs(m), sn(m), y(m);
  int iters = 0;
  bcs_status status = BCS_OK;
  KrylovState* ks = reinterpret_cast<KrylovState*>(s->kst.p);
  for (;;) {
    BCS_OKR(scale_copy(s, 1.0 / beta, r, V, N));
    bool breakdown = false;
    if (dev) {
      BCS_OKR(ks_init(s, ks, beta, bnorm, iters, m, cfg.maxiter, cfg.tol));
      if (!s->kry_exec) {
        BCS_OKR(capture_cycle(s, ks));
        s->kry_key[0] = s->kv.p;
        s->kry_key[1] = s->kz.p;
        s->kry_key[2] = s->kw.p;
        s->kry_key[3] = s->kt.p;
        s->kry_key[4] = s->kvj.p;
        s->kry_m = m;
      }
      BCS_CU(s, cudaGraphLaunch(s->kry_exec, s->stream));
      BCS_OKR(ks_finish_cycle(s, ks, Z, zf, x, N));
      // true residual, its norm and the cycle's outcome in one read
      BCS_OKR(spmv64(s, s->lv[0].A, x, false, r, b, K_SPMV64));
      BCS_OKR(dot(s, r, r, N, SLOT_N));
      BCS_OKR(ks_export(s, ks, SLOT_S));
      BCS_OKR(fetch_scalars(s, SLOT_S + 3));
      const int it_now = (int)s->hscal[SLOT_S];
      count_steps(s, it_now - iters);
      iters = it_now;
      breakdown = (int)s->hscal[SLOT_S + 2] == KS_BREAKDOWN;
      beta = std::sqrt(s->hscal[SLOT_N]);
    } else {
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      int jend = 0;
      for (int j = 0; j < m; ++j) {
        double* w = V + (size_t)(j + 1) * N;
        void* zj = Z + (size_t)j * N * zbytes(s);
        BCS_OKR(apply_M(s, V + (size_t)j * N, zj, N));
        BCS_OKR(apply_A(s, zj, w, N));
        // pass 1 also yields ||w||^2 (w is vector j+1 of V); pass 2's
        // update also yields the new ||w||^2
        BCS_OKR(multidot(s, V, N, j + 2, w, N, SLOT_A));
        BCS_OKR(gs_update(s, V, N, j + 1, s->scal.p + SLOT_A, w, N));
        BCS_OKR(multidot(s, V, N, j + 1, w, N, SLOT_B));
        BCS_OKR(gs_update_norm(s, V, N, j + 1, s->scal.p + SLOT_B, w, N, SLOT_N));
        BCS_OKR(fetch_scalars(s, SLOT_N + 1));
        const double* hs = s->hscal;
        const double wn0 = std::sqrt(hs[SLOT_A + j + 1]);
        const double hn = std::sqrt(hs[SLOT_N]);
        for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hs[SLOT_A + i] + hs[SLOT_B + i];
        H[(size_t)(j + 1) * m + j] = hn;
        for (int i = 0; i < j; ++i) {
          const double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
          H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
          H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
        }
        const double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
        if (c == 0.0) {
          cs[j] = 1.0;
          sn[j] = 0.0;
        } else {
          const double d = std::sqrt(a * a + c * c);
          cs[j] = a / d;
          sn[j] = c / d;
        }
        H[(size_t)j * m + j] = cs[j] * a + sn[j] * c;
        H[(size_t)(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        ++iters;
        jend = j + 1;
        if (!std::isfinite(hn) || !std::isfinite(g[j + 1])) {
          breakdown = true;
          break;
        }
        if (!(hn > 1e-14 * wn0)) break;  // happy breakdown: no v_{j+1}
        BCS_OKR(scale_copy(s, 1.0 / hn, w, w, N));
        if (std::fabs(g[j + 1]) <= cfg.tol * bnorm || iters >= cfg.maxiter) break;
      }
      for (int i = jend - 1; i >= 0; --i) {
        double t = g[i];
        for (int k = i + 1; k < jend; ++k) t -= H[(size_t)i * m + k] * y[k];
        y[i] = t / H[(size_t)i * m + i];
      }
      if (!breakdown) BCS_OKR(add_combination(s, Z, zf, N, jend, y.data(), x, N));
      BCS_OKR(true_residual(s, b, x, r, N, &beta));
    }
    res->rel_res_final = beta / bnorm;
    if (breakdown || !std::isfinite(beta)) {
      status = BCS_BREAKDOWN;
      break;
    }
    if (beta <= cfg.tol * bnorm) {
      status = BCS_OK;
      break;
    }
    if (iters >= cfg.maxiter) {
      status = BCS_NOT_CONVERGED;
      break;
    }
    res->restarts++;
  }
  res->iters = iters;
  return status;
}

// ---- device-resident BiCGStab --------------------------------------------------
// One BiCGStab iteration (dots, the rho / alpha / omega scalars and their
// tests in kernels, the vector updates, two preconditioner applications and
// products) is captured once into a graph WHILE body; the loop runs until
// something happens that the host must act on (a breakdown restart, a small
// residual to confirm on the true residual, omega = 0, the iteration
// limit). The host then does exactly what the host-driven loop does at that
// point, so both loops give the same iterates.

// z = M^{-1} v with every launch capturable (no nested graph launch).
bcs_status apply_M_plain(Solver* s, const double* v, void* z, size_t N) {
  const int pc = s->setup_cfg.precond;
  Level& L0 = s->lv[0];
  if (s->setup_cfg.precision == BCS_PREC_FP64) {
    if (pc == BCS_PC_AMG) return precond_cycle64(s, v, (double*)z);
    return sgs_fixed(s, v, z);
  }
  BCS_OKR(cast_vec<double, float>(s, v, (float*)L0.vb.p, N));
  if (pc == BCS_PC_AMG) {
    BCS_OKR(precond_cycle32(s, (const float*)L0.vb.p, (float*)L0.vx.p));
    BCS_CU(s, cudaMemcpyAsync(z, L0.vx.p, N * sizeof(float), cudaMemcpyDeviceToDevice, s->stream));
    return BCS_OK;
  }
  return sgs_fixed(s, L0.vb.p, z);
}

bcs_status bicg_iteration_dev(Solver* s, BicgState* bs, cudaGraphConditionalHandle cond) {
  const size_t N = (size_t)s->C * s->n;
  const bool zf = cycle_is_float(s);
  double *r = s->kv.p, *rhat = r + N, *p = r + 2 * N, *v = r + 3 * N, *sv = r + 4 * N, *t = r + 5 * N;
  void* ph = s->kz.p;
  void* sh = s->kz.p + N * zbytes(s);
  BCS_OKR(dot(s, rhat, r, N, SLOT_A));
  BCS_OKR(bs_rho(s, bs));
  BCS_OKR(bs_p_update(s, bs, r, v, p, N));
  BCS_OKR(apply_M_plain(s, p, ph, N));
  BCS_OKR(apply_A(s, ph, v, N));
  BCS_OKR(dot(s, rhat, v, N, SLOT_A));
  BCS_OKR(bs_alpha(s, bs));
  BCS_OKR(bs_s_update(s, bs, r, v, sv, N));
  BCS_OKR(dot(s, sv, sv, N, SLOT_N));
  BCS_OKR(bs_snorm(s, bs));
  BCS_OKR(apply_M_plain(s, sv, sh, N));
  BCS_OKR(apply_A(s, sh, t, N));
  BCS_OKR(multidot(s, sv, N, 2, t, N, SLOT_A));  // (s, t), (t, t)
  BCS_OKR(bs_omega(s, bs));
  BCS_OKR(bs_x_update(s, bs, ph, zf, s->kx_dev, N));
  BCS_OKR(bs_r_update(s, bs, sv, t, r, N));
  BCS_OKR(dot(s, r, r, N, SLOT_N));
  return bs_end(s, bs, cond);
}

bcs_status capture_bicg(Solver* s, BicgState* bs) {
  long long kl[BCS_NUM_KERNEL_KINDS];
  double kb[BCS_NUM_KERNEL_KINDS], kf[BCS_NUM_KERNEL_KINDS];
  const long long l0 = s->launches;
  for (int k = 0; k < BCS_NUM_KERNEL_KINDS; ++k) {
    kl[k] = s->kind_launches[k];
    kb[k] = s->kind_bytes[k];
    kf[k] = s->kind_flops[k];
  }
  if (!s->gstream) BCS_CU(s, cudaStreamCreateWithFlags(&s->gstream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  BCS_CU(s, cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle cond = 0;
  cudaGraphNode_t node = nullptr;
  cudaGraphNodeParams prm{};
  cudaError_t e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = cond;
    prm.conditional.type = cudaGraphCondTypeWhile;
    prm.conditional.size = 1;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &prm);
  }
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(s->gstream, prm.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return s->fail(BCS_ECUDA, std::string("BiCGStab loop graph: ") + cudaGetErrorString(e));
  }
  const cudaStream_t own = s->stream;
  s->stream = s->gstream;
  const bcs_status st = bicg_iteration_dev(s, bs, cond);
  s->stream = own;
  cudaGraph_t captured = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(s->gstream, &captured);
  s->launches = l0;
  for (int k = 0; k < BCS_NUM_KERNEL_KINDS; ++k) {
    s->bcg_kind_launches[k] = s->kind_launches[k] - kl[k];
    s->bcg_kind_bytes[k] = s->kind_bytes[k] - kb[k];
    s->bcg_kind_flops[k] = s->kind_flops[k] - kf[k];
    s->kind_launches[k] = kl[k];
    s->kind_bytes[k] = kb[k];
    s->kind_flops[k] = kf[k];
  }
  if (st != BCS_OK || ce != cudaSuccess) {
    cudaGraphDestroy(g);
    if (st != BCS_OK) return st;
    return s->fail(BCS_ECUDA, std::string("BiCGStab loop capture: ") + cudaGetErrorString(ce));
  }
  const cudaError_t ie = cudaGraphInstantiate(&s->bcg_exec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    s->bcg_exec = nullptr;
    return s->fail(BCS_ECUDA, std::string("BiCGStab loop instantiate: ") + cudaGetErrorString(ie));
  }
  return BCS_OK;
}

bcs_status bicgstab_dev(Solver* s, const double* b, double* x, bcs_result* res) {
  const bcs_config& cfg = s->cfg;
  const size_t N = (size_t)s->C * s->n;
  const bool zf = cycle_is_float(s);
  BCS_ALLOC(s, s->kv, (size_t)6 * N);
  BCS_ALLOC(s, s->kz, (size_t)2 * N * zbytes(s));
  BCS_ALLOC(s, s->kst, std::max(sizeof(KrylovState), sizeof(BicgState)));
  BCS_ALLOC(s, s->red, (size_t)72 * 1184);
  if (zf) BCS_ALLOC(s, s->kt, N);
  if (s->bcg_exec && (s->bcg_key[0] != (const void*)s->kv.p || s->bcg_key[1] != (const void*)s->kz.p ||
                      s->bcg_key[2] != (const void*)x)) {
    cudaGraphExecDestroy(s->bcg_exec);
    s->bcg_exec = nullptr;
  }
  double *r = s->kv.p, *rhat = r + N;
  void* ph = s->kz.p;
  const double tol = cfg.tol;
  double bnorm = 0.0, rn = 0.0;
  BCS_OKR(initial_residual(s, b, x, r, N, &bnorm, &rn));
  res->iters = 0;
  res->restarts = 0;
  if (bnorm == 0.0) {
    BCS_CU(s, cudaMemsetAsync(x, 0, N * sizeof(double), s->stream));
    res->rel_res_initial = res->rel_res_final = 0.0;
    return BCS_OK;
  }
  res->rel_res_initial = res->rel_res_final = rn / bnorm;
  if (!std::isfinite(rn)) return BCS_BREAKDOWN;
  if (rn <= tol * bnorm) return BCS_OK;
  BCS_CU(s, cudaMemcpyAsync(rhat, r, N * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
  BicgState* bs = reinterpret_cast<BicgState*>(s->kst.p);
  BCS_OKR(bs_init(s, bs, 0, cfg.maxiter, tol, bnorm, 2));
  s->kx_dev = x;
  if (!s->bcg_exec) {
    BCS_OKR(capture_bicg(s, bs));
    s->bcg_key[0] = s->kv.p;
    s->bcg_key[1] = s->kz.p;
    s->bcg_key[2] = x;
  }
  bool restarted = false;
  int it = 0;
  bcs_status status = BCS_NOT_CONVERGED;
  // restart from the true residual (the host loop's restart); false when a
  // breakdown recurs
  auto restart = [&](bool breakdown, bool* ok) -> bcs_status {
    *ok = true;
    if (breakdown) {
      if (restarted) {
        *ok = false;
        return BCS_OK;
      }
      restarted = true;
    }
    double tr = 0.0;
    BCS_OKR(true_residual(s, b, x, r, N, &tr));
    BCS_CU(s, cudaMemcpyAsync(rhat, r, N * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    res->restarts++;
    return bs_init(s, bs, it, cfg.maxiter, tol, bnorm, 1);
  };
  while (it < cfg.maxiter) {
    BCS_CU(s, cudaGraphLaunch(s->bcg_exec, s->stream));
    BCS_OKR(bs_export(s, bs));
    BCS_OKR(fetch_scalars(s, SLOT_S + 3));
    const int it_now = (int)s->hscal[SLOT_S];
    const int stop = (int)s->hscal[SLOT_S + 1];
    const double alpha = s->hscal[SLOT_S + 2];
    for (int k = 0; k < BCS_NUM_KERNEL_KINDS; ++k) {  // the executed iterations' launches
      const int steps = std::max(1, it_now - it);
      s->launches += s->bcg_kind_launches[k] * steps;
      s->kind_launches[k] += s->bcg_kind_launches[k] * steps;
      s->kind_bytes[k] += s->bcg_kind_bytes[k] * steps;
      s->kind_flops[k] += s->bcg_kind_flops[k] * steps;
    }
    it = it_now;
    bool ok = true;
    if (stop == BS_BREAK || stop == BS_OMEGA0) {
      BCS_OKR(restart(true, &ok));
      if (!ok) {
        status = BCS_BREAKDOWN;
        break;
      }
      continue;
    }
    if (stop == BS_S_SMALL || stop == BS_R_SMALL) {
      if (stop == BS_S_SMALL) BCS_OKR(add_combination(s, ph, zf, N, 1, &alpha, x, N));
      double tr = 0.0;
      BCS_OKR(true_residual(s, b, x, r, N, &tr));
      if (tr <= tol * bnorm) {
        status = BCS_OK;
        break;
      }
      BCS_OKR(restart(false, &ok));
      continue;
    }
    break;  // BS_MAXITER
  }
  double tr = 0.0;
  BCS_OKR(true_residual(s, b, x, s->kv.p, N, &tr));
  res->rel_res_final = tr / bnorm;
  if (status == BCS_NOT_CONVERGED && res->rel_res_final <= tol) status = BCS_OK;
  if (status == BCS_NOT_CONVERGED && !std::isfinite(tr)) status = BCS_BREAKDOWN;
  res->iters = it;
  return status;
}

bcs_status bicgstab(Solver* s, const double* b, double* x, bcs_result* res) {
  const bcs_config& cfg = s->cfg;
  const size_t N = (size_t)s->C * s->n;
  const bool zf = cycle_is_float(s);
  BCS_ALLOC(s, s->kv, (size_t)6 * N);
  BCS_ALLOC(s, s->kz, (size_t)2 * N * zbytes(s));
  double *r = s->kv.p, *rhat = r + N, *p = r + 2 * N, *v = r + 3 * N, *sv = r + 4 * N, *t = r + 5 * N;
  void* ph = s->kz.p;
  void* sh = s->kz.p + N * zbytes(s);
  const double tol = cfg.tol;
  double bnorm = 0.0, rn = 0.0;
  BCS_OKR(initial_residual(s, b, x, r, N, &bnorm, &rn));
  res->iters = 0;
  res->restarts = 0;
  if (bnorm == 0.0) {
    BCS_CU(s, cudaMemsetAsync(x, 0, N * sizeof(double), s->stream));
    res->rel_res_initial = res->rel_res_final = 0.0;
    return BCS_OK;
  }
  res->rel_res_initial = res->rel_res_final = rn / bnorm;
  if (!std::isfinite(rn)) return BCS_BREAKDOWN;
  if (rn <= tol * bnorm) return BCS_OK;
  BCS_CU(s, cudaMemcpyAsync(rhat, r, N * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
  double rho_old = 1.0, alpha = 1.0, omega = 1.0;
  bool first = true, restarted = false;
  int it = 0;
  bcs_status status = BCS_NOT_CONVERGED;
  // restart from the true residual; false when a breakdown recurs
  auto restart = [&](bool breakdown, bool* ok) -> bcs_status {
    *ok = true;
    if (breakdown) {
      if (restarted) {
        *ok = false;
        return BCS_OK;
      }
      restarted = true;
    }
    double tr = 0.0;
    BCS_OKR(true_residual(s, b, x, r, N, &tr));
    BCS_CU(s, cudaMemcpyAsync(rhat, r, N * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    first = true;
    res->restarts++;
    return BCS_OK;
  };
  bool ok = true;
  while (it < cfg.maxiter) {
    BCS_OKR(dot(s, rhat, r, N, SLOT_A));
    BCS_OKR(fetch_scalars(s, 1));
    const double rho = s->hscal[0];
    if (rho == 0.0 || !std::isfinite(rho)) {
      BCS_OKR(restart(true, &ok));
      if (!ok) {
        status = BCS_BREAKDOWN;
        break;
      }
      continue;
    }
    if (first) {
      BCS_CU(s, cudaMemcpyAsync(p, r, N * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    } else {
      const double beta = (rho / rho_old) * (alpha / omega);
      BCS_OKR(bicg_p_update(s, beta, omega, r, v, p, N));
    }
    first = false;
    BCS_OKR(apply_M(s, p, ph, N));
    BCS_OKR(apply_A(s, ph, v, N));
    BCS_OKR(dot(s, rhat, v, N, SLOT_A));
    BCS_OKR(fetch_scalars(s, 1));
    const double den = s->hscal[0];
    if (den == 0.0 || !std::isfinite(den)) {
      BCS_OKR(restart(true, &ok));
      if (!ok) {
        status = BCS_BREAKDOWN;
        break;
      }
      continue;
    }
    alpha = rho / den;
    BCS_CU(s, cudaMemcpyAsync(sv, r, N * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    BCS_OKR(axpby(s, -alpha, v, 1.0, sv, N));
    ++it;
    double snrm = 0.0;
    BCS_OKR(norm(s, sv, N, &snrm));
    if (snrm <= tol * bnorm) {
      BCS_OKR(add_combination(s, ph, zf, N, 1, &alpha, x, N));
      double tr = 0.0;
      BCS_OKR(true_residual(s, b, x, r, N, &tr));
      if (tr <= tol * bnorm) {
        status = BCS_OK;
        break;
      }
      BCS_OKR(restart(false, &ok));
      continue;
    }
    BCS_OKR(apply_M(s, sv, sh, N));
    BCS_OKR(apply_A(s, sh, t, N));
    BCS_OKR(multidot(s, sv, N, 2, t, N, SLOT_A));  // (s, t), (t, t)
    BCS_OKR(fetch_scalars(s, 2));
    const double ts = s->hscal[0], tt = s->hscal[1];
    if (tt == 0.0 || !std::isfinite(tt)) {
      BCS_OKR(restart(true, &ok));
      if (!ok) {
        status = BCS_BREAKDOWN;
        break;
      }
      continue;
    }
    omega = ts / tt;
    {
      const double coef[2] = {alpha, omega};
      BCS_OKR(add_combination(s, ph, zf, N, 2, coef, x, N));  // ph and sh are consecutive
    }
    BCS_CU(s, cudaMemcpyAsync(r, sv, N * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    BCS_OKR(axpby(s, -omega, t, 1.0, r, N));
    rho_old = rho;
    BCS_OKR(norm(s, r, N, &rn));
    if (rn <= tol * bnorm) {
      double tr = 0.0;
      BCS_OKR(true_residual(s, b, x, r, N, &tr));
      if (tr <= tol * bnorm) {
        status = BCS_OK;
        break;
      }
      BCS_OKR(restart(false, &ok));
      continue;
    }
    if (omega == 0.0) {
      BCS_OKR(restart(true, &ok));
      if (!ok) {
        status = BCS_BREAKDOWN;
        break;
      }
    }
  }
  double tr = 0.0;
  BCS_OKR(true_residual(s, b, x, s->kv.p, N, &tr));
  res->rel_res_final = tr / bnorm;
  if (status == BCS_NOT_CONVERGED && res->rel_res_final <= tol) status = BCS_OK;
  if (status == BCS_NOT_CONVERGED && !std::isfinite(tr)) status = BCS_BREAKDOWN;
  res->iters = it;
  return status;
}

}  // namespace

bcs_status solve(Solver* s, const double* b, double* x, bcs_result* res) {
  const auto t0 = std::chrono::steady_clock::now();
  const long long syncs0 = s->host_syncs;
  bcs_status st = s->cfg.solver == BCS_BICGSTAB ? (device_cycle_ok(s) ? bicgstab_dev(s, b, x, res) : bicgstab(s, b, x, res))
                                                : fgmres(s, b, x, res);
  if (st == BCS_ECUDA || st == BCS_ENOMEM || st == BCS_EINVAL) return st;
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return s->fail(BCS_ECUDA, std::string("solve: ") + cudaGetErrorString(e));
  res->status = st;
  res->host_syncs = (int)(s->host_syncs - syncs0 + 1);
  res->levels = (int)s->lv.size();
  res->setup_ms = s->last_setup_ms;
  res->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (st == BCS_NOT_CONVERGED) s->err = "maximum iterations reached above the tolerance";
  if (st == BCS_BREAKDOWN) s->err = "Krylov breakdown or non-finite residual";
  return st;
}


// ---- batched FGMRES ------------------------------------------------------------
// Several systems (uneven sizes, same block size and cycle options) solved
// in lockstep: each restart round is one launch of a graph whose WHILE body
// is one Arnoldi step of every live case (batched kernels, blockIdx.z =
// case), followed by the round's back substitutions, x updates, true
// residuals and one read of every case's outcome. A case leaves the round
// when its own stop test fires and the batch when it has converged, broken
// down or reached maxiter. Each case's arithmetic is the single-system
// device loop's, so its iterates equal those of solving it alone.
namespace {

bcs_status capture_batch(Solver* s0, const BCase* cases, const std::vector<BCase>& host, int count, int m,
                         size_t maxN, int max_rows, cudaGraphExec_t* exec, long long* body_launches) {
  if (!s0->gstream) BCS_CU(s0, cudaStreamCreateWithFlags(&s0->gstream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  BCS_CU(s0, cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle cond = 0;
  cudaGraphNode_t node = nullptr;
  cudaGraphNodeParams prm{};
  cudaError_t e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = cond;
    prm.conditional.type = cudaGraphCondTypeWhile;
    prm.conditional.size = 1;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &prm);
  }
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(s0->gstream, prm.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return s0->fail(BCS_ECUDA, std::string("batched loop graph: ") + cudaGetErrorString(e));
  }
  const long long l0 = s0->launches;
  const cudaStream_t own = s0->stream;
  s0->stream = s0->gstream;
  bcs_status st = kb_step_begin(s0, cases, count);
  if (st == BCS_OK) st = kb_take_vj(s0, cases, count, maxN);
  if (st == BCS_OK) st = kb_cycle(s0, cases, host, count);
  if (st == BCS_OK) st = kb_store_z(s0, cases, count, maxN);
  if (st == BCS_OK) st = kb_spmv_w(s0, cases, count, max_rows);
  if (st == BCS_OK) st = kb_multidot(s0, cases, count, true, m + 1, SLOT_A);
  if (st == BCS_OK) st = kb_gs_update(s0, cases, count, SLOT_A, -1);
  if (st == BCS_OK) st = kb_multidot(s0, cases, count, false, m, SLOT_B);
  if (st == BCS_OK) st = kb_gs_update(s0, cases, count, SLOT_B, SLOT_N);
  if (st == BCS_OK) st = kb_givens(s0, cases, count, cond);
  if (st == BCS_OK) st = kb_scale_next(s0, cases, count, maxN);
  s0->stream = own;
  cudaGraph_t captured = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(s0->gstream, &captured);
  *body_launches = s0->launches - l0;
  s0->launches = l0;
  if (st != BCS_OK || ce != cudaSuccess) {
    cudaGraphDestroy(g);
    if (st != BCS_OK) return st;
    return s0->fail(BCS_ECUDA, std::string("batched loop capture: ") + cudaGetErrorString(ce));
  }
  const cudaError_t ie = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    *exec = nullptr;
    return s0->fail(BCS_ECUDA, std::string("batched loop instantiate: ") + cudaGetErrorString(ie));
  }
  return BCS_OK;
}

}  // namespace

bcs_status solve_batch(Solver* const* ss, int count, const double* const* b, double* const* x, bcs_result* res) {
  Solver* s0 = ss[0];
  const int m = s0->cfg.restart;
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<BCase> host(count);
  std::vector<double> bnorm(count, 0.0), beta(count, 0.0);
  std::vector<int> iters(count, 0), active(count, 0);
  std::vector<bcs_status> status(count, BCS_OK);
  size_t maxN = 0;
  int max_rows = 0;
  for (int i = 0; i < count; ++i) {
    Solver* s = ss[i];
    const size_t N = (size_t)s->C * s->n;
    BCS_ALLOC(s, s->kv, (size_t)(m + 1) * N);
    BCS_ALLOC(s, s->kz, (size_t)m * N * sizeof(float));
    BCS_ALLOC(s, s->kr, N);
    BCS_ALLOC(s, s->kw, N);
    BCS_ALLOC(s, s->kt, N);
    BCS_ALLOC(s, s->kst, sizeof(KrylovState));
    BCS_ALLOC(s, s->red, (size_t)72 * 1184);
    BCS_OKR(initial_residual(s, b[i], x[i], s->kr.p, N, &bnorm[i], &beta[i]));  // synchronises s's stream
    res[i] = bcs_result{};
    res[i].rel_res_initial = res[i].rel_res_final = bnorm[i] > 0.0 ? beta[i] / bnorm[i] : 0.0;
    res[i].levels = (int)s->lv.size();
    res[i].setup_ms = s->last_setup_ms;
    if (bnorm[i] == 0.0) {
      BCS_CU(s, cudaMemsetAsync(x[i], 0, N * sizeof(double), s->stream));
      BCS_CU(s, cudaStreamSynchronize(s->stream));
    } else if (!std::isfinite(beta[i])) {
      status[i] = BCS_BREAKDOWN;
    } else if (beta[i] > s->cfg.tol * bnorm[i]) {
      active[i] = 1;
    }
    BCase& h = host[i];
    std::memset(&h, 0, sizeof(h));
    h.n_levels = (int)s->lv.size();
    h.rows = s->C;
    h.N = N;
    h.ks = reinterpret_cast<KrylovState*>(s->kst.p);
    h.V = s->kv.p;
    h.w = s->kw.p;
    h.kt = s->kt.p;
    h.scal = s->scal.p;
    h.red = s->red.p;
    h.x = x[i];
    h.r = s->kr.p;
    h.b = b[i];
    h.Z = reinterpret_cast<float*>(s->kz.p);
    h.rp = s->lv[0].A.rp.p;
    h.ci = s->lv[0].A.ci.p;
    h.val = s->lv[0].A.v.p;
    h.cinv = s->cinv.p;
    h.cN = s->lv.back().coarse_kind == 0 ? s->cN : 0;
    for (int l = 0; l < h.n_levels; ++l) {
      const Level& L = s->lv[l];
      BLevel& t = h.lv[l];
      t.rows = L.A.rows;
      t.nslices = L.nslices;
      t.smap = L.smap;
      t.nagg = L.nagg;
      t.coarse_kind = L.coarse_kind;
      t.rp = L.A.rp.p;
      t.srow = L.srow.p;
      t.sptr = L.sptr.p;
      t.sci = L.sci.p;
      t.mptr = L.mptr.p;
      t.mem = L.mem.p;
      t.agg = L.agg.p;
      t.sv = s->setup_cfg.precision == BCS_PREC_FP32 ? (const void*)L.s32.p : (const void*)L.s16.p;
      t.dinv = L.dinv32.p;
      t.vb = (float*)L.vb.p;
      t.vx = (float*)L.vx.p;
      t.vr = (float*)L.vr.p;
      t.vt = (float*)L.vt.p;
    }
    maxN = std::max(maxN, N);
    max_rows = std::max(max_rows, s->C);
  }
  // device tables: cases | live flags | round flags | outcomes
  DBuf<char> buf;
  const size_t off_live = ((size_t)count * sizeof(BCase) + 255) / 256 * 256;
  const size_t off_round = off_live + ((size_t)count * sizeof(int) + 255) / 256 * 256;
  const size_t off_out = off_round + ((size_t)count * sizeof(int) + 255) / 256 * 256;
  BCS_ALLOC(s0, buf, off_out + (size_t)count * 4 * sizeof(double));
  int* live = reinterpret_cast<int*>(buf.p + off_live);
  int* round = reinterpret_cast<int*>(buf.p + off_round);
  double* out = reinterpret_cast<double*>(buf.p + off_out);
  for (int i = 0; i < count; ++i) {
    host[i].live = live + i;
    host[i].round = round + i;
  }
  const BCase* cases = reinterpret_cast<const BCase*>(buf.p);
  BCS_CU(s0, cudaMemcpyAsync(buf.p, host.data(), (size_t)count * sizeof(BCase), cudaMemcpyHostToDevice, s0->stream));
  BCS_CU(s0, cudaMemsetAsync(live, 0, (size_t)count * sizeof(int), s0->stream));
  // every case starts stopped; the ones with work are started per round
  for (int i = 0; i < count; ++i) BCS_CU(s0, cudaMemsetAsync(ss[i]->kst.p, 0xff, sizeof(KrylovState), s0->stream));
  cudaGraphExec_t exec = nullptr;
  long long body = 0;
  std::vector<double> h_out((size_t)count * 4);
  bcs_status st = BCS_OK;
  for (;;) {
    bool any = false;
    for (int i = 0; i < count; ++i) any |= active[i] != 0;
    if (!any) break;
    int prev_iters = 0;
    for (int i = 0; i < count; ++i) {
      if (!active[i]) continue;
      Solver* s = ss[i];
      const size_t N = host[i].N;
      st = scale_copy(s0, 1.0 / beta[i], host[i].r, host[i].V, N);
      if (st == BCS_OK) st = ks_init(s0, host[i].ks, beta[i], bnorm[i], iters[i], m, s->cfg.maxiter, s->cfg.tol);
      if (st != BCS_OK) break;
      prev_iters = std::max(prev_iters, iters[i]);
    }
    if (st != BCS_OK) break;
    BCS_CU(s0, cudaMemcpyAsync(round, active.data(), (size_t)count * sizeof(int), cudaMemcpyHostToDevice, s0->stream));
    if (!exec) {
      st = capture_batch(s0, cases, host, count, m, maxN, max_rows, &exec, &body);
      if (st != BCS_OK) break;
    }
    if (cudaGraphLaunch(exec, s0->stream) != cudaSuccess) {
      st = s0->fail(BCS_ECUDA, "batched loop launch failed");
      break;
    }
    st = kb_finish(s0, cases, count, maxN);
    if (st == BCS_OK) st = kb_resid_r(s0, cases, count, max_rows);
    if (st == BCS_OK) st = kb_norm_r(s0, cases, count);
    if (st == BCS_OK) st = kb_gather_out(s0, cases, count, out);
    if (st != BCS_OK) break;
    if (cudaMemcpyAsync(h_out.data(), out, h_out.size() * sizeof(double), cudaMemcpyDeviceToHost, s0->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(s0->stream) != cudaSuccess) {
      st = s0->fail(BCS_ECUDA, "batched solve: reading the round's outcome failed");
      break;
    }
    int steps = 0;
    for (int i = 0; i < count; ++i) {
      if (!active[i]) continue;
      Solver* s = ss[i];
      const int it = (int)h_out[4 * i + 1];
      steps = std::max(steps, it - iters[i]);
      iters[i] = it;
      beta[i] = std::sqrt(h_out[4 * i]);
      res[i].rel_res_final = beta[i] / bnorm[i];
      const bool breakdown = (int)h_out[4 * i + 3] == KS_BREAKDOWN;
      if (breakdown || !std::isfinite(beta[i])) {
        status[i] = BCS_BREAKDOWN;
        active[i] = 0;
      } else if (beta[i] <= s->cfg.tol * bnorm[i]) {
        status[i] = BCS_OK;
        active[i] = 0;
      } else if (iters[i] >= s->cfg.maxiter) {
        status[i] = BCS_NOT_CONVERGED;
        active[i] = 0;
      } else {
        res[i].restarts++;
      }
    }
    s0->launches += body * steps;
    (void)prev_iters;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (st != BCS_OK) return st;
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  for (int i = 0; i < count; ++i) {
    res[i].host_syncs = 1 + res[i].restarts + (iters[i] > 0 ? 1 : 0);  // initial residual, one read per round
    res[i].iters = iters[i];
    res[i].status = status[i];
    res[i].solve_ms = ms;
  }
  return BCS_OK;
}

}  // namespace bcs
