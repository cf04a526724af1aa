// FP64 CPU oracle: assembly of the density-based coupled system from a cell
// flow state and face geometry (Sec. 2.1, Eqs. approxJac1 / approxJac2 and
// the pseudo-time linearisation of Eq. discretBackward).
//
// TEST INFRASTRUCTURE ONLY (see oracle.h). Plain loops over the faces in
// ascending order; nothing here is shared with the CUDA library.
//
// Readings (the paper cites Luo et al. and Blazek for the details):
//   * Q = (rho, rho u, rho v, rho w, rho E), ideal gas:
//     p = (gamma - 1) (rho E - rho |u|^2 / 2), H = (rho E + p) / rho,
//     c^2 = gamma p / rho.
//   * J(Q, n) is the Jacobian dF/dQ of the inviscid normal flux
//     F(Q, n) = (rho V, rho u V + p n, rho H V), V = u . n, written out in
//     closed form; it is linear in n, so J(Q, -n) = -J(Q, n).
//   * lambda of face (i, j) = spectral radius of the Roe matrix at the Roe
//     average of Q_i and Q_j, |u~ . n| + c~, plus the viscous spectral radius
//     max(4/3, gamma) mu / (Pr rho~ d) (d = distance between the cell
//     centres, rho~ = sqrt(rho_i rho_j)).
//   * Face f with owner i, neighbour j, unit normal n from i to j, area S:
//       A_ii += S/2 (J(Q_i, n) + lambda I)      (Eq. approxJac1)
//       A_ij  = S/2 (J(Q_j, n) - lambda I)      (Eq. approxJac2)
//     and, seen from j (R_ji(n_ji) = -R_ij(n_ij), n_ji = -n):
//       A_jj += S/2 (-J(Q_j, n) + lambda I),  A_ji = S/2 (-J(Q_i, n) - lambda I).
//   * Pseudo-time term V/dtau I with the local step dtau_c = CFL V_c /
//     sum_f lambda_f S_f over the faces of c, i.e. (sum_f lambda_f S_f / CFL) I,
//     added to A_cc after the face terms.
//   * upper[f] holds A_ij (row owner), lower[f] A_ji (row neighbour), as the
//     solver's LDU input.
#include <cmath>
#include <cstdint>
#include <vector>

#include "oracle.h"

namespace {

struct State {
  double rho, u, v, w, E, p, H, c2;
};

bool state_of(const double* Q, double gamma, State& s) {
  s.rho = Q[0];
  if (!(s.rho > 0.0)) return false;
  s.u = Q[1] / s.rho;
  s.v = Q[2] / s.rho;
  s.w = Q[3] / s.rho;
  s.E = Q[4] / s.rho;
  const double q2 = s.u * s.u + s.v * s.v + s.w * s.w;
  s.p = (gamma - 1.0) * (Q[4] - 0.5 * s.rho * q2);
  if (!(s.p > 0.0)) return false;
  s.H = (Q[4] + s.p) / s.rho;
  s.c2 = gamma * s.p / s.rho;
  return true;
}

void flux_jacobian(const State& s, const double* n, double gamma, double* J) {
  const double g1 = gamma - 1.0, g2 = gamma - 2.0;
  const double V = s.u * n[0] + s.v * n[1] + s.w * n[2];
  const double phi = 0.5 * g1 * (s.u * s.u + s.v * s.v + s.w * s.w);
  const double vel[3] = {s.u, s.v, s.w};
  // continuity row: d(rho V)/dQ
  J[0] = 0.0;
  J[1] = n[0];
  J[2] = n[1];
  J[3] = n[2];
  J[4] = 0.0;
  // momentum rows a = x, y, z: d(rho u_a V + p n_a)/dQ
  for (int a = 0; a < 3; ++a) {
    double* r = J + 5 * (1 + a);
    r[0] = phi * n[a] - vel[a] * V;
    for (int b = 0; b < 3; ++b) r[1 + b] = vel[a] * n[b] - g1 * vel[b] * n[a];
    r[1 + a] = V - g2 * vel[a] * n[a];
    r[4] = g1 * n[a];
  }
  // energy row: d(rho H V)/dQ
  J[20] = V * (phi - s.H);
  for (int b = 0; b < 3; ++b) J[21 + b] = s.H * n[b] - g1 * vel[b] * V;
  J[24] = gamma * V;
}

bool face_lambda(const double* Qo, const double* Qn, const double* n, double d, double gamma, double mu,
                 double prandtl, double* lam) {
  State a, b;
  if (!state_of(Qo, gamma, a) || !state_of(Qn, gamma, b)) return false;
  const double ra = std::sqrt(a.rho), rb = std::sqrt(b.rho), rs = ra + rb;
  const double u = (ra * a.u + rb * b.u) / rs;
  const double v = (ra * a.v + rb * b.v) / rs;
  const double w = (ra * a.w + rb * b.w) / rs;
  const double H = (ra * a.H + rb * b.H) / rs;
  const double c2 = (gamma - 1.0) * (H - 0.5 * (u * u + v * v + w * w));
  if (!(c2 > 0.0)) return false;
  const double rho = ra * rb;
  const double lc = std::fabs(u * n[0] + v * n[1] + w * n[2]) + std::sqrt(c2);
  const double lv = std::fmax(4.0 / 3.0, gamma) * mu / (prandtl * rho * d);
  *lam = lc + lv;
  return true;
}

}  // namespace

extern "C" {

int or_euler_flux(const double* Q, const double* n, double gamma, double* F) {
  State s;
  if (!state_of(Q, gamma, s)) return 1;
  const double V = s.u * n[0] + s.v * n[1] + s.w * n[2];
  F[0] = s.rho * V;
  F[1] = Q[1] * V + s.p * n[0];
  F[2] = Q[2] * V + s.p * n[1];
  F[3] = Q[3] * V + s.p * n[2];
  F[4] = s.rho * s.H * V;
  return 0;
}

int or_flux_jacobian(const double* Q, const double* n, double gamma, double* J) {
  State s;
  if (!state_of(Q, gamma, s)) return 1;
  flux_jacobian(s, n, gamma, J);
  return 0;
}

int or_face_lambda(const double* Qo, const double* Qn, const double* n, double d, double gamma, double mu,
                   double prandtl, double* lam) {
  return face_lambda(Qo, Qn, n, d, gamma, mu, prandtl, lam) ? 0 : 1;
}

int or_assemble_density(int C, int F, const int32_t* owner, const int32_t* nb, const double* Q,
                        const double* area, const double* normal, const double* dist, double gamma, double mu,
                        double prandtl, double cfl, double* diag, double* upper, double* lower) {
  if (!(gamma > 1.0) || !(mu >= 0.0) || !(prandtl > 0.0) || !(cfl > 0.0)) return 1;
  std::vector<State> st(C);
  for (int c = 0; c < C; ++c)
    if (!state_of(Q + 5 * (size_t)c, gamma, st[c])) return 1;
  std::vector<double> tsum(C, 0.0);
  for (size_t e = 0; e < (size_t)C * 25; ++e) diag[e] = 0.0;
  for (int f = 0; f < F; ++f) {
    const int i = owner[f], j = nb[f];
    const double* n = normal + 3 * (size_t)f;
    const double S = area[f];
    if (!(S >= 0.0) || !(dist[f] > 0.0)) return 1;
    double lam = 0.0;
    if (!face_lambda(Q + 5 * (size_t)i, Q + 5 * (size_t)j, n, dist[f], gamma, mu, prandtl, &lam)) return 1;
    double Ji[25], Jj[25];
    flux_jacobian(st[i], n, gamma, Ji);
    flux_jacobian(st[j], n, gamma, Jj);
    const double h = 0.5 * S;
    double* Di = diag + 25 * (size_t)i;
    double* Dj = diag + 25 * (size_t)j;
    double* U = upper + 25 * (size_t)f;
    double* L = lower + 25 * (size_t)f;
    for (int r = 0; r < 5; ++r)
      for (int c = 0; c < 5; ++c) {
        const int e = 5 * r + c;
        const double I = r == c ? lam : 0.0;
        Di[e] += h * (Ji[e] + I);
        U[e] = h * (Jj[e] - I);
        Dj[e] += h * (-Jj[e] + I);
        L[e] = h * (-Ji[e] - I);
      }
    tsum[i] += lam * S;
    tsum[j] += lam * S;
  }
  for (int c = 0; c < C; ++c)
    for (int r = 0; r < 5; ++r) diag[25 * (size_t)c + 6 * r] += tsum[c] / cfl;
  return 0;
}

}  // extern "C"
