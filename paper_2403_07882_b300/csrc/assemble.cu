// Assembly of the density-based coupled system on the device (Sec. 2.1,
// Eqs. approxJac1 / approxJac2, pseudo-time term of Eq. discretBackward).
//
// Q = (rho, rho u, rho v, rho w, rho E) per cell, ideal gas with ratio gamma.
// J(Q, n) is the Jacobian of the inviscid normal flux
// (rho V, rho u V + p n, rho H V), V = u . n; it is linear in n. For a face
// with unit normal n from cell i to cell j, area S and spectral radius lambda
// (Roe average of the two states plus max(4/3, gamma) mu / (Pr rho~ d)):
//   A_ii += S/2 (J(Q_i, n) + lambda I),   A_ij = S/2 (J(Q_j, n) - lambda I)
// and, from j's side with n_ji = -n, A_jj += S/2 (J(Q_j, -n) + lambda I),
// A_ji = S/2 (J(Q_i, -n) - lambda I). The pseudo-time term is
// V/dtau = sum_f lambda_f S_f / CFL (local step dtau = CFL V / sum lambda S).
//
// Work split: k_face_lambda computes lambda once per face; k_assemble_cells
// takes one cell c per thread and, for each face of c with c's outward
// normal n_c, evaluates M = J(Q_c, S/2 n_c) once: the block of column c in
// the other cell's row is -M - S/2 lambda I, and (J being linear in n) the
// cell's own block is J(Q_c, sum_f S/2 n_c) + sum_f S/2 lambda (1 + 2/CFL) I,
// one more Jacobian per cell instead of a sum of one per face. Every block is
// written by exactly one thread; results equal the face-by-face sums up to
// rounding.
#include "internal.h"

namespace bcs {
namespace {

struct Gas {
  double rho, vel[3], H, phi;  // phi = (gamma - 1) |u|^2 / 2
};

__device__ __forceinline__ bool gas_of(const double* __restrict__ Q, double gamma, Gas& g) {
  const double rho = __ldg(Q), m0 = __ldg(Q + 1), m1 = __ldg(Q + 2), m2 = __ldg(Q + 3), rE = __ldg(Q + 4);
  g.rho = rho;
  const double ir = 1.0 / rho;
  g.vel[0] = m0 * ir;
  g.vel[1] = m1 * ir;
  g.vel[2] = m2 * ir;
  const double q2 = g.vel[0] * g.vel[0] + g.vel[1] * g.vel[1] + g.vel[2] * g.vel[2];
  const double p = (gamma - 1.0) * (rE - 0.5 * rho * q2);
  g.phi = 0.5 * (gamma - 1.0) * q2;
  g.H = (rE + p) * ir;
  return rho > 0.0 && p > 0.0;  // false for NaN too
}

// out = sgn * J(Q, n) + shift * I (n need not be a unit vector).
__device__ __forceinline__ void put_jacobian(double* __restrict__ out, const Gas& g, const double n[3], double gamma,
                                             double sgn, double shift) {
  const double g1 = gamma - 1.0;
  const double V = g.vel[0] * n[0] + g.vel[1] * n[1] + g.vel[2] * n[2];
  out[0] = shift;
  out[1] = sgn * n[0];
  out[2] = sgn * n[1];
  out[3] = sgn * n[2];
  out[4] = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double* row = out + 5 * (a + 1);
    row[0] = sgn * (g.phi * n[a] - g.vel[a] * V);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      // d(rho u_a V + p n_a)/d(rho u_b)
      const double jab = (a == b) ? V + g.vel[a] * n[a] - g1 * g.vel[a] * n[a] : g.vel[a] * n[b] - g1 * g.vel[b] * n[a];
      row[b + 1] = sgn * jab + (a == b ? shift : 0.0);
    }
    row[4] = sgn * g1 * n[a];
  }
  out[20] = sgn * V * (g.phi - g.H);
#pragma unroll
  for (int b = 0; b < 3; ++b) out[21 + b] = sgn * (g.H * n[b] - g1 * g.vel[b] * V);
  out[24] = sgn * gamma * V + shift;
}

// lambda per face; flag bit 1: a non-physical state or geometry.
__global__ void k_face_lambda(int F, const int32_t* __restrict__ pos_up, const int32_t* __restrict__ pos_lo,
                              const int32_t* __restrict__ ci, const double* __restrict__ Q,
                              const double* __restrict__ area, const double* __restrict__ normal,
                              const double* __restrict__ dist, double gamma, double visc, double* __restrict__ lam,
                              int32_t* __restrict__ flag) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const int i = __ldg(ci + __ldg(pos_lo + f)), j = __ldg(ci + __ldg(pos_up + f));
  Gas a, b;
  const bool ok = gas_of(Q + (size_t)i * 5, gamma, a) & gas_of(Q + (size_t)j * 5, gamma, b);
  const double ra = sqrt(a.rho), rb = sqrt(b.rho), irs = 1.0 / (ra + rb);
  double un = 0.0, q2 = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double uk = (ra * a.vel[k] + rb * b.vel[k]) * irs;
    un += uk * __ldg(normal + (size_t)f * 3 + k);
    q2 += uk * uk;
  }
  const double H = (ra * a.H + rb * b.H) * irs;
  const double c2 = (gamma - 1.0) * (H - 0.5 * q2);
  const double d = __ldg(dist + f), S = __ldg(area + f);
  if (!ok || !(c2 > 0.0) || !(d > 0.0) || !(S >= 0.0)) atomicOr(flag, 1);
  lam[f] = fabs(un) + sqrt(c2) + visc / (ra * rb * d);
}

// One thread per cell (see the file comment). BSR: blocks go to the solver's
// block-CSR values; otherwise to the LDU arrays diag / upper / lower.
template <bool BSR>
__global__ void __launch_bounds__(128) k_assemble_cells(
    int C, const int32_t* __restrict__ rp, const int32_t* __restrict__ src, const int32_t* __restrict__ pos_diag,
    const int32_t* __restrict__ pos_up, const int32_t* __restrict__ pos_lo, const double* __restrict__ Q,
    const double* __restrict__ area, const double* __restrict__ normal, const double* __restrict__ lam, double gamma,
    double inv_cfl, double* __restrict__ diag, double* __restrict__ upper, double* __restrict__ lower,
    double* __restrict__ val, int32_t* __restrict__ flag) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  Gas g;
  if (!gas_of(Q + (size_t)c * 5, gamma, g)) atomicOr(flag, 1);
  double N[3] = {0.0, 0.0, 0.0};
  double hl = 0.0;
  for (int p = __ldg(rp + c), pe = __ldg(rp + c + 1); p < pe; ++p) {
    const int code = __ldg(src + p);
    if (code < 0) continue;  // the diagonal block
    const int f = code >> 1;
    const bool own = (code & 1) == 0;  // c is the face's owner
    const double hs = 0.5 * __ldg(area + f);
    const double hn = own ? hs : -hs;
    const double n[3] = {hn * __ldg(normal + (size_t)f * 3), hn * __ldg(normal + (size_t)f * 3 + 1),
                         hn * __ldg(normal + (size_t)f * 3 + 2)};
    const double hsl = hs * __ldg(lam + f);
    double* out;
    if (BSR)
      out = val + (size_t)__ldg((own ? pos_lo : pos_up) + f) * 25;
    else
      out = (own ? lower : upper) + (size_t)f * 25;
    put_jacobian(out, g, n, gamma, -1.0, -hsl);
    N[0] += n[0];
    N[1] += n[1];
    N[2] += n[2];
    hl += hsl;
  }
  double* od = BSR ? val + (size_t)__ldg(pos_diag + c) * 25 : diag + (size_t)c * 25;
  put_jacobian(od, g, N, gamma, 1.0, hl + 2.0 * hl * inv_cfl);
}

}  // namespace

bcs_status assemble_density(Solver* s, const double* Q, const double* area, const double* normal, const double* dist,
                            const bcs_flow_params& prm, double* diag, double* upper, double* lower) {
  const int C = s->C, F = s->F;
  const Bsr& A = s->lv[0].A;
  const bool bsr = !diag;
  if (bsr) BCS_ALLOC(s, s->lv[0].A.v, (size_t)A.nnz * 25);
  DBuf<double> lam;
  BCS_ALLOC(s, lam, F > 0 ? F : 1);
  BCS_CU(s, cudaMemsetAsync(s->flag.p, 0, sizeof(int32_t), s->stream));
  const double visc = (prm.gamma > 4.0 / 3.0 ? prm.gamma : 4.0 / 3.0) * prm.mu / prm.prandtl;
  if (F > 0)
    BCS_LAUNCH(s, K_ASSEMBLE, 104.0 * F, 0, k_face_lambda, grid_for(F, 256), 256, 0, F, s->pos_up.p, s->pos_lo.p,
               A.ci.p, Q, area, normal, dist, prm.gamma, visc, lam.p, s->flag.p);
  const double bytes = 40.0 * C + 48.0 * 2 * F + 8.0 * F + 200.0 * (C + 2.0 * F);
  const double flops = 2 * F * 60.0 + C * 60.0;
  if (bsr)
    BCS_LAUNCH(s, K_ASSEMBLE, bytes, flops, k_assemble_cells<true>, grid_for(C, 128), 128, 0, C, A.rp.p, s->src.p,
               s->pos_diag.p, s->pos_up.p, s->pos_lo.p, Q, area, normal, lam.p, prm.gamma, 1.0 / prm.cfl, nullptr,
               nullptr, nullptr, s->lv[0].A.v.p, s->flag.p);
  else
    BCS_LAUNCH(s, K_ASSEMBLE, bytes, flops, k_assemble_cells<false>, grid_for(C, 128), 128, 0, C, A.rp.p, s->src.p,
               s->pos_diag.p, s->pos_up.p, s->pos_lo.p, Q, area, normal, lam.p, prm.gamma, 1.0 / prm.cfl, diag,
               upper, lower, nullptr, s->flag.p);
  int32_t h = 0;
  BCS_CU(s, cudaMemcpyAsync(&h, s->flag.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  if (h & 1) return s->fail(BCS_EINVAL, "assembly: a state with rho <= 0 or p <= 0, or area < 0 or dist <= 0");
  return BCS_OK;
}

}  // namespace bcs
