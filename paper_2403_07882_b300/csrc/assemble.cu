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
// Work split: k_cell_prims turns each cell's state into (sqrt(rho), u, v, w,
// H) once (the only division and square root per cell); k_face_lambda
// computes lambda once per face from the two cells' primitives;
// k_assemble_cells takes one cell c per thread and, for each face of c with
// c's outward normal n_c, evaluates M = J(Q_c, S/2 n_c) once: the block of
// column c in the other cell's row is -M - S/2 lambda I, and (J being linear
// in n) the cell's own block is J(Q_c, sum_f S/2 n_c) + sum_f S/2 lambda
// (1 + 2/CFL) I, one more Jacobian per cell instead of a sum of one per face.
// A warp's 32 blocks of one face slot are staged in shared memory and
// written out as whole 200-byte blocks. Every block is written by exactly
// one thread; results equal the face-by-face sums up to rounding.
#include "internal.h"

namespace bcs {
namespace {

struct Gas {
  double rho, vel[3], H, phi;  // phi = (gamma - 1) |u|^2 / 2
};

constexpr int AS_WARPS = 4;
constexpr int AS_NN = 25;

// prim[c] = (sqrt(rho), u, v, w, H) of row c (the caller's cell perm[c] when
// the cells are renumbered); flag bit 1 for rho <= 0 or p <= 0 (or NaN)
__global__ void k_cell_prims(int C, const double* __restrict__ Q, const int32_t* __restrict__ perm, double gamma,
                             double* __restrict__ prim, int32_t* __restrict__ flag) {
  dep_enter();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const double* q = Q + (size_t)(perm ? perm[c] : c) * 5;
  const double rho = __ldg(q), rE = __ldg(q + 4);
  const double ir = 1.0 / rho;
  const double u = __ldg(q + 1) * ir, v = __ldg(q + 2) * ir, w = __ldg(q + 3) * ir;
  const double p = (gamma - 1.0) * (rE - 0.5 * rho * (u * u + v * v + w * w));
  if (!(rho > 0.0 && p > 0.0)) atomicOr(flag, 1);
  double* o = prim + (size_t)c * 5;
  o[0] = sqrt(rho);
  o[1] = u;
  o[2] = v;
  o[3] = w;
  o[4] = (rE + p) * ir;
}

__device__ __forceinline__ Gas gas_of(const double* __restrict__ prim, int c, double gamma) {
  Gas g;
  const double* q = prim + (size_t)c * 5;
  const double sr = __ldg(q);
  g.rho = sr * sr;
  g.vel[0] = __ldg(q + 1);
  g.vel[1] = __ldg(q + 2);
  g.vel[2] = __ldg(q + 3);
  g.H = __ldg(q + 4);
  g.phi = 0.5 * (gamma - 1.0) * (g.vel[0] * g.vel[0] + g.vel[1] * g.vel[1] + g.vel[2] * g.vel[2]);
  return g;
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

// lambda per face; flag bit 1: a non-physical Roe state or geometry.
__global__ void k_face_lambda(int F, const int32_t* __restrict__ pos_up, const int32_t* __restrict__ pos_lo,
                              const int32_t* __restrict__ ci, const double* __restrict__ prim,
                              const double* __restrict__ normal, const double* __restrict__ area,
                              const double* __restrict__ dist, double gamma, double visc, double* __restrict__ lam,
                              int32_t* __restrict__ flag) {
  dep_enter();
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const double* a = prim + (size_t)__ldg(ci + __ldg(pos_lo + f)) * 5;
  const double* b = prim + (size_t)__ldg(ci + __ldg(pos_up + f)) * 5;
  const double ra = __ldg(a), rb = __ldg(b), d = __ldg(dist + f), S = __ldg(area + f);
  // one division for both 1 / (ra + rb) and visc / (ra rb d)
  const double den = (ra + rb) * (ra * rb * d);
  const double r = 1.0 / den;
  const double irs = r * (ra * rb * d), ivd = r * (ra + rb);
  double un = 0.0, q2 = 0.0;
#pragma unroll
  for (int k = 1; k <= 3; ++k) {
    const double uk = (ra * __ldg(a + k) + rb * __ldg(b + k)) * irs;
    un += uk * __ldg(normal + (size_t)f * 3 + k - 1);
    q2 += uk * uk;
  }
  const double H = (ra * __ldg(a + 4) + rb * __ldg(b + 4)) * irs;
  const double c2 = (gamma - 1.0) * (H - 0.5 * q2);
  if (!(c2 > 0.0) || !(d > 0.0) || !(S >= 0.0) || !(ra > 0.0) || !(rb > 0.0)) atomicOr(flag, 1);
  lam[f] = fabs(un) + sqrt(c2) + visc * ivd;
}

// One thread per cell (see the file comment). BSR: blocks go to the solver's
// block-CSR values; otherwise to the LDU arrays diag / upper / lower. Each
// face slot's 32 blocks pass through the warp's shared-memory stage so that
// the stores are whole blocks.
template <bool BSR>
__global__ void __launch_bounds__(AS_WARPS * 32) k_assemble_cells(
    int C, const int32_t* __restrict__ rp, const int32_t* __restrict__ src, const int32_t* __restrict__ pos_up, const int32_t* __restrict__ pos_lo, const double* __restrict__ prim,
    const double* __restrict__ area, const double* __restrict__ normal, const double* __restrict__ lam, double gamma,
    double inv_cfl, double* __restrict__ diag, double* __restrict__ upper, double* __restrict__ lower,
    double* __restrict__ val) {
  dep_enter();
  __shared__ double stage_s[AS_WARPS][32 * AS_NN];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* stage = stage_s[warp];
  double* mine = stage + lane * AS_NN;  // odd stride: no bank conflicts
  const int c = (blockIdx.x * AS_WARPS + warp) * 32 + lane;
  const bool live = c < C;
  if (__all_sync(0xffffffffu, !live)) return;
  Gas g{};
  int p0 = 0, p1 = 0;
  if (live) {
    g = gas_of(prim, c, gamma);
    p0 = __ldg(rp + c);
    p1 = __ldg(rp + c + 1);
  }
  // a warp-uniform number of face slots: the most faces of a cell in the
  // warp (every row holds its diagonal block once)
  const int slots = __reduce_max_sync(0xffffffffu, live ? p1 - p0 - 1 : 0);
  double N[3] = {0.0, 0.0, 0.0};
  double hl = 0.0;
  int p = p0, pd = -1, cd = -1;  // diagonal block: position, caller's cell
  for (int k = 0; k <= slots; ++k) {
    double* dest = nullptr;
    if (k < slots) {
      // next off-diagonal block of this row, if any
      int code = -1;
      while (p < p1 && (code = __ldg(src + p)) < 0) {
        pd = p;
        cd = -1 - code;
        ++p;
      }
      if (p < p1) {
        ++p;
        const int f = code >> 1;
        const bool own = (code & 1) == 0;  // c is the face's owner
        const double hs = 0.5 * __ldg(area + f);
        const double hn = own ? hs : -hs;
        const double n[3] = {hn * __ldg(normal + (size_t)f * 3), hn * __ldg(normal + (size_t)f * 3 + 1),
                             hn * __ldg(normal + (size_t)f * 3 + 2)};
        const double hsl = hs * __ldg(lam + f);
        put_jacobian(mine, g, n, gamma, -1.0, -hsl);
        N[0] += n[0];
        N[1] += n[1];
        N[2] += n[2];
        hl += hsl;
        dest = BSR ? val + (size_t)__ldg((own ? pos_lo : pos_up) + f) * AS_NN
                   : (own ? lower : upper) + (size_t)f * AS_NN;
      }
    } else if (live) {
      // a row whose diagonal comes after all its faces: find it now
      for (; pd < 0 && p < p1; ++p) {
        const int code = __ldg(src + p);
        if (code < 0) {
          pd = p;
          cd = -1 - code;
        }
      }
      put_jacobian(mine, g, N, gamma, 1.0, hl + 2.0 * hl * inv_cfl);
      dest = BSR ? val + (size_t)pd * AS_NN : diag + (size_t)cd * AS_NN;
    }
    __syncwarp();
    // write the staged blocks: element i of the warp's 32 x 25 stage
    for (int i = lane; i < 32 * AS_NN; i += 32) {
      const int j = i / AS_NN;
      double* dj = (double*)__shfl_sync(0xffffffffu, (unsigned long long)dest, j);
      if (dj) dj[i - j * AS_NN] = stage[i];
    }
    __syncwarp();
  }
}

}  // namespace

bcs_status assemble_density(Solver* s, const double* Q, const double* area, const double* normal, const double* dist,
                            const bcs_flow_params& prm, double* diag, double* upper, double* lower) {
  const int C = s->C, F = s->F;
  const Bsr& A = s->lv[0].A;
  const bool bsr = !diag;
  if (bsr) BCS_ALLOC(s, s->lv[0].A.v, (size_t)A.nnz * 25);
  DBuf<double> lam, prim;
  BCS_ALLOC(s, lam, F > 0 ? F : 1);
  BCS_ALLOC(s, prim, (size_t)C * 5);
  BCS_CU(s, cudaMemsetAsync(s->flag.p, 0, sizeof(int32_t), s->stream));
  const double visc = (prm.gamma > 4.0 / 3.0 ? prm.gamma : 4.0 / 3.0) * prm.mu / prm.prandtl;
  BCS_LAUNCH_DEP(s, K_ASSEMBLE, 80.0 * C, 0, k_cell_prims, grid_for(C, 256), 256, 0, C, Q,
             s->reordered ? (const int32_t*)s->perm.p : nullptr, prm.gamma, prim.p, s->flag.p);
  if (F > 0)
    BCS_LAUNCH_DEP(s, K_ASSEMBLE, 104.0 * F, 0, k_face_lambda, grid_for(F, 256), 256, 0, F, s->pos_up.p, s->pos_lo.p,
               A.ci.p, prim.p, normal, area, dist, prm.gamma, visc, lam.p, s->flag.p);
  // prim, per face side area + normal + lambda + LDU code, blocks written
  const double bytes = 40.0 * C + 44.0 * 2 * F + 200.0 * (C + 2.0 * F);
  const double flops = 2 * F * 55.0 + C * 60.0;
  const unsigned grid = grid_for(C, AS_WARPS * 32);
  if (bsr)
    BCS_LAUNCH_DEP(s, K_ASSEMBLE, bytes, flops, k_assemble_cells<true>, grid, AS_WARPS * 32, 0, C, A.rp.p, s->src.p,
               s->pos_up.p, s->pos_lo.p, prim.p, area, normal, lam.p, prm.gamma, 1.0 / prm.cfl,
               nullptr, nullptr, nullptr, s->lv[0].A.v.p);
  else
    BCS_LAUNCH_DEP(s, K_ASSEMBLE, bytes, flops, k_assemble_cells<false>, grid, AS_WARPS * 32, 0, C, A.rp.p, s->src.p,
               s->pos_up.p, s->pos_lo.p, prim.p, area, normal, lam.p, prm.gamma, 1.0 / prm.cfl, diag,
               upper, lower, nullptr);
  int32_t h = 0;
  BCS_CU(s, cudaMemcpyAsync(&h, s->flag.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
  BCS_CU(s, cudaStreamSynchronize(s->stream));
  if (h & 1) return s->fail(BCS_EINVAL, "assembly: a state with rho <= 0 or p <= 0, or area < 0 or dist <= 0");
  return BCS_OK;
}

}  // namespace bcs
