// FP64 CPU oracle for the block-coupled solve. TEST INFRASTRUCTURE ONLY:
// loaded by the tests, the package smoke check and the benchmark's CPU
// baseline; never by the product path. Plain, sequential, no shared code with
// the CUDA library. Build: g++ -O2 -ffp-contract=off (no implicit FMA; every
// fused multiply-add below is an explicit std::fma that is part of the
// definition). See oracle.h for what each function follows.
#include "oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <utility>
#include <vector>

namespace {

struct Bsr {
  int rows = 0, cols = 0, n = 0;
  std::vector<int32_t> rp, ci;
  std::vector<double> v;
  int nnz() const { return rp.empty() ? 0 : rp[rows]; }
  const double* blk(int k) const { return v.data() + (size_t)k * n * n; }
  double* blk(int k) { return v.data() + (size_t)k * n * n; }
};

// Position of column j in row i, or -1 (rows are sorted ascending).
int find_in_row(const Bsr& A, int i, int j) {
  int lo = A.rp[i], hi = A.rp[i + 1];
  for (int k = lo; k < hi; ++k)
    if (A.ci[k] == j) return k;
  return -1;
}

// T = X * Y for n x n row-major blocks; each T[r][c] accumulates over m in
// ascending order with fma, starting from +0.
void block_mul(int n, const double* X, const double* Y, double* T) {
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      double acc = 0.0;
      for (int m = 0; m < n; ++m) acc = std::fma(X[r * n + m], Y[m * n + c], acc);
      T[r * n + c] = acc;
    }
}

}  // namespace

extern "C" {

void or_config_default(or_config* c) {
  c->solver = 0;
  c->restart = 30;
  c->tol = 1e-8;
  c->maxiter = 1000;
  c->precond = 0;
  c->pmode = 1;
  c->matching_rounds = 4;
  c->agg_passes = 2;
  c->jacobi_omega = 0.8;
  c->nu1 = 2;
  c->nu2 = 2;
  c->coarse_size = 32;
  c->max_levels = 20;
  c->max_coarsen_ratio = 0.8;
  c->p_omega = 4.0 / 3.0;
  c->coarse_dense_max = 1024;
  c->coarse_sweeps = 8;
  c->smoother = 0;
}

// ---------------------------------------------------------------------------
// LDU addressing and the LDU -> block-CSR map (Eq. 1; Sec. 2.3; Alg. 1).
// ---------------------------------------------------------------------------
int or_ldu_check(int C, int F, const int32_t* owner, const int32_t* nb) {
  if (C < 1 || F < 0) return 1;
  std::vector<std::pair<int, int>> pairs((size_t)F);
  for (int f = 0; f < F; ++f) {
    int o = owner[f], m = nb[f];
    if (o < 0 || o >= C || m < 0 || m >= C || o == m) return 1;
    pairs[f] = {std::min(o, m), std::max(o, m)};
  }
  std::sort(pairs.begin(), pairs.end());
  for (int f = 1; f < F; ++f)
    if (pairs[f] == pairs[f - 1]) return 1;
  return 0;
}

int or_ldu_structure(int C, int F, const int32_t* owner, const int32_t* nb,
                     int32_t* row_ptr, int32_t* col, int32_t* pos_diag, int32_t* pos_up,
                     int32_t* pos_lo) {
  int bad = or_ldu_check(C, F, owner, nb);
  if (bad) return bad;
  // Each row lists (column, source); source = 0: diagonal, 1 + f: upper[f]
  // (row owner), -1 - f: lower[f] (row neighbour).
  std::vector<std::vector<std::pair<int, long>>> rows((size_t)C);
  for (int i = 0; i < C; ++i) rows[i].push_back({i, 0});
  for (int f = 0; f < F; ++f) {
    rows[owner[f]].push_back({nb[f], 1L + f});
    rows[nb[f]].push_back({owner[f], -1L - f});
  }
  int p = 0;
  row_ptr[0] = 0;
  for (int i = 0; i < C; ++i) {
    std::sort(rows[i].begin(), rows[i].end());
    for (auto& e : rows[i]) {
      col[p] = e.first;
      if (e.second == 0) pos_diag[i] = p;
      else if (e.second > 0) pos_up[e.second - 1] = p;
      else pos_lo[-e.second - 1] = p;
      ++p;
    }
    row_ptr[i + 1] = p;
  }
  return 0;
}

void or_ldu_values(int C, int F, int n, const int32_t* pos_diag, const int32_t* pos_up,
                   const int32_t* pos_lo, const double* diag, const double* upper,
                   const double* lower, double* val) {
  size_t nn = (size_t)n * n;
  for (int i = 0; i < C; ++i) std::memcpy(val + pos_diag[i] * nn, diag + i * nn, nn * 8);
  for (int f = 0; f < F; ++f) {
    std::memcpy(val + pos_up[f] * nn, upper + f * nn, nn * 8);
    std::memcpy(val + pos_lo[f] * nn, lower + f * nn, nn * 8);
  }
}

void or_bsr_to_ldu(int C, int F, int n, const int32_t* pos_diag, const int32_t* pos_up,
                   const int32_t* pos_lo, const double* val, double* diag, double* upper,
                   double* lower) {
  size_t nn = (size_t)n * n;
  for (int i = 0; i < C; ++i) std::memcpy(diag + i * nn, val + pos_diag[i] * nn, nn * 8);
  for (int f = 0; f < F; ++f) {
    std::memcpy(upper + f * nn, val + pos_up[f] * nn, nn * 8);
    std::memcpy(lower + f * nn, val + pos_lo[f] * nn, nn * 8);
  }
}

// y_i = sum_j A_ij x_j, Eq. 1's left-hand side.
void or_bsr_spmv(int rows, int n, const int32_t* rp, const int32_t* ci, const double* val,
                 const double* x, double* y) {
  size_t nn = (size_t)n * n;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < rows; ++i)
    for (int r = 0; r < n; ++r) {
      double acc = 0.0;
      for (int k = rp[i]; k < rp[i + 1]; ++k) {
        const double* a = val + k * nn + r * n;
        const double* xj = x + (size_t)ci[k] * n;
        for (int c = 0; c < n; ++c) acc += a[c] * xj[c];
      }
      y[(size_t)i * n + r] = acc;
    }
}

// Gauss-Jordan on [A | I] with implicit partial pivoting and deferred
// normalisation. Step k picks, among rows not yet used as pivots, the largest
// |M[i][k]| (first such row on ties), takes its reciprocal r = 1 / pivot, then
// for every other row i computes l = M[i][k] * r and
// M[i][j] = fma(-l, M[p][j], M[i][j]) for j >= k. Finally
// inv[k][:] = M[p_k][N:] * (1 / M[p_k][k]).
int or_dense_inverse(int N, const double* A, double* inv) {
  const size_t W = 2 * (size_t)N;
  std::vector<double> M((size_t)N * W, 0.0);
  for (int i = 0; i < N; ++i) {
    for (int j = 0; j < N; ++j) M[i * W + j] = A[(size_t)i * N + j];
    M[i * W + N + i] = 1.0;
  }
  std::vector<char> used(N, 0);
  std::vector<int> prow(N);
  for (int k = 0; k < N; ++k) {
    int p = -1;
    double best = -1.0;
    for (int i = 0; i < N; ++i) {
      if (used[i]) continue;
      double a = std::fabs(M[i * W + k]);
      if (a > best) { best = a; p = i; }
    }
    double piv = M[p * W + k];
    if (piv == 0.0) return 1;
    used[p] = 1;
    prow[k] = p;
    const double rpiv = 1.0 / piv;
    for (int i = 0; i < N; ++i) {
      if (i == p) continue;
      double l = M[i * W + k] * rpiv;
      for (size_t j = k; j < W; ++j) M[i * W + j] = std::fma(-l, M[p * W + j], M[i * W + j]);
    }
  }
  for (int k = 0; k < N; ++k) {
    int p = prow[k];
    const double rd = 1.0 / M[p * W + k];
    for (int j = 0; j < N; ++j) inv[(size_t)k * N + j] = M[p * W + N + j] * rd;
  }
  return 0;
}

void or_block_norms(int nblocks, int n, const double* val, double* nrm) {
  size_t nn = (size_t)n * n;
  for (int k = 0; k < nblocks; ++k) {
    double acc = 0.0;
    for (size_t e = 0; e < nn; ++e) acc = std::fma(val[k * nn + e], val[k * nn + e], acc);
    nrm[k] = std::sqrt(acc);
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Aggregation AMG (Sec. 2.3: aggregation for block systems built from graph
// matching). The paper does not state the rule; the reading implemented here:
//  * edge weight from block Frobenius norms
//      w_ij = (N(A_ij) + N(A_ji)) / (2 max(N(A_ii), N(A_jj)))   (0 if the max is 0)
//  * synchronous handshake rounds: every unmatched row picks its unmatched
//    neighbour of largest positive weight (smaller index on ties); mutual
//    picks become pairs; at most matching_rounds rounds
//  * an unmatched row with a matched neighbour of positive weight joins the
//    aggregate of the strongest such neighbour; the rest stay singletons
//  * aggregates are numbered by ascending smallest member row
//  * later passes repeat this on the Galerkin product with the tentative
//    prolongation (block sums), and compose the maps.
// ---------------------------------------------------------------------------
namespace {

// C = A * B (block sparse). Row i's columns are the sorted union of B's rows
// k for k in A's row i; C_ij[r][c] accumulates, for k in ascending order of
// A's row, then m ascending, fma(A_ik[r][m], B_kj[m][c], acc).
void spgemm(const Bsr& A, const Bsr& B, Bsr& Cm) {
  const int n = A.n, nn = n * n;
  Cm.rows = A.rows;
  Cm.cols = B.cols;
  Cm.n = n;
  Cm.rp.assign(A.rows + 1, 0);
  Cm.ci.clear();
  for (int i = 0; i < A.rows; ++i) {
    std::vector<int> cols;
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      int j = A.ci[k];
      for (int kk = B.rp[j]; kk < B.rp[j + 1]; ++kk) cols.push_back(B.ci[kk]);
    }
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    Cm.ci.insert(Cm.ci.end(), cols.begin(), cols.end());
    Cm.rp[i + 1] = (int32_t)Cm.ci.size();
  }
  Cm.v.assign((size_t)Cm.nnz() * nn, 0.0);
  for (int i = 0; i < A.rows; ++i) {
    for (int q = Cm.rp[i]; q < Cm.rp[i + 1]; ++q) {
      int J = Cm.ci[q];
      double* acc = Cm.blk(q);
      for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
        int kk = find_in_row(B, A.ci[k], J);
        if (kk < 0) continue;
        const double* a = A.blk(k);
        const double* bb = B.blk(kk);
        for (int r = 0; r < n; ++r)
          for (int c = 0; c < n; ++c)
            for (int m = 0; m < n; ++m) acc[r * n + c] = std::fma(a[r * n + m], bb[m * n + c], acc[r * n + c]);
      }
    }
  }
}

// R = P^T (blocks transposed), rows of R list P's rows in ascending order.
void transpose(const Bsr& P, Bsr& R) {
  const int n = P.n, nn = n * n;
  R.rows = P.cols;
  R.cols = P.rows;
  R.n = n;
  R.rp.assign(R.rows + 1, 0);
  for (int k = 0; k < P.nnz(); ++k) R.rp[P.ci[k] + 1]++;
  for (int J = 0; J < R.rows; ++J) R.rp[J + 1] += R.rp[J];
  R.ci.assign(P.nnz(), 0);
  R.v.assign((size_t)P.nnz() * nn, 0.0);
  std::vector<int> cur(R.rp.begin(), R.rp.end() - 1);
  for (int i = 0; i < P.rows; ++i)
    for (int k = P.rp[i]; k < P.rp[i + 1]; ++k) {
      int q = cur[P.ci[k]]++;
      R.ci[q] = i;
      for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) R.v[(size_t)q * nn + r * n + c] = P.v[(size_t)k * nn + c * n + r];
    }
}

Bsr tentative_P(int rows, int n, const std::vector<int32_t>& agg, int nagg) {
  Bsr P;
  P.rows = rows;
  P.cols = nagg;
  P.n = n;
  P.rp.resize(rows + 1);
  P.ci.resize(rows);
  P.v.assign((size_t)rows * n * n, 0.0);
  for (int i = 0; i < rows; ++i) {
    P.rp[i] = i;
    P.ci[i] = agg[i];
    for (int r = 0; r < n; ++r) P.v[(size_t)i * n * n + r * n + r] = 1.0;
  }
  P.rp[rows] = rows;
  return P;
}

// Galerkin product R A P with R = P^T: first AP = A P, then R (AP).
void galerkin(const Bsr& A, const Bsr& P, Bsr& R, Bsr& AP, Bsr& Ac) {
  transpose(P, R);
  spgemm(A, P, AP);
  spgemm(R, AP, Ac);
}

// Galerkin product with the piecewise-constant (tentative) P: block (I, J)
// of P^T A P is the sum of the fine blocks A_ij with agg(i) = I and
// agg(j) = J, taken directly from its definition: rows i of aggregate I in
// ascending order, each row's blocks in ascending column order, a plain
// left-to-right FP64 sum from +0. Columns of row I: the sorted aggregates
// of its rows' columns.
void galerkin_tentative(const Bsr& A, const std::vector<int32_t>& agg, int nagg, Bsr& Ac) {
  const int n = A.n, nn = n * n;
  std::vector<std::vector<int>> members(nagg);
  for (int i = 0; i < A.rows; ++i) members[agg[i]].push_back(i);
  Ac.rows = Ac.cols = nagg;
  Ac.n = n;
  Ac.rp.assign(nagg + 1, 0);
  Ac.ci.clear();
  for (int I = 0; I < nagg; ++I) {
    std::vector<int> cols;
    for (int i : members[I])
      for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) cols.push_back(agg[A.ci[k]]);
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    Ac.ci.insert(Ac.ci.end(), cols.begin(), cols.end());
    Ac.rp[I + 1] = (int32_t)Ac.ci.size();
  }
  Ac.v.assign((size_t)Ac.nnz() * nn, 0.0);
  for (int I = 0; I < nagg; ++I)
    for (int q = Ac.rp[I]; q < Ac.rp[I + 1]; ++q) {
      const int J = Ac.ci[q];
      double* acc = Ac.blk(q);
      for (int i : members[I])
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
          if (agg[A.ci[k]] != J) continue;
          for (int e = 0; e < nn; ++e) acc[e] = acc[e] + A.blk(k)[e];
        }
    }
}

// One matching pass on the graph of A, weights from block norms.
int match_pass(const Bsr& A, const or_config& cfg, std::vector<int32_t>& agg) {
  const int C = A.rows, nnz = A.nnz();
  std::vector<double> nrm(nnz);
  or_block_norms(nnz, A.n, A.v.data(), nrm.data());
  std::vector<int> dpos(C);
  for (int i = 0; i < C; ++i) dpos[i] = find_in_row(A, i, i);
  std::vector<double> w(nnz, 0.0);
  for (int i = 0; i < C; ++i)
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      int j = A.ci[k];
      if (j == i) continue;
      int kt = find_in_row(A, j, i);
      double s = nrm[k] + (kt >= 0 ? nrm[kt] : 0.0);
      double di = dpos[i] >= 0 ? nrm[dpos[i]] : 0.0;
      double dj = dpos[j] >= 0 ? nrm[dpos[j]] : 0.0;
      double d = 2.0 * (di < dj ? dj : di);
      w[k] = d > 0.0 ? s / d : 0.0;
    }
  std::vector<int> mate(C, -1), choice(C, -1);
  for (int round = 0; round < cfg.matching_rounds; ++round) {
    for (int i = 0; i < C; ++i) {
      choice[i] = -1;
      if (mate[i] >= 0) continue;
      double bw = 0.0;
      for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
        int j = A.ci[k];
        if (j == i || mate[j] >= 0) continue;
        if (w[k] > bw) { bw = w[k]; choice[i] = j; }
      }
    }
    bool any = false;
    for (int i = 0; i < C; ++i)
      if (mate[i] < 0 && choice[i] >= 0 && choice[choice[i]] == i) { mate[i] = choice[i]; any = true; }
    if (!any) break;
  }
  std::vector<int> root(C);
  for (int i = 0; i < C; ++i) {
    if (mate[i] >= 0) { root[i] = std::min(i, mate[i]); continue; }
    int best = -1;
    double bw = 0.0;
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      int j = A.ci[k];
      if (j == i || mate[j] < 0) continue;
      if (w[k] > bw) { bw = w[k]; best = j; }
    }
    root[i] = best >= 0 ? std::min(best, mate[best]) : i;
  }
  std::vector<int> amin(C, C);
  for (int i = 0; i < C; ++i) amin[root[i]] = std::min(amin[root[i]], i);
  std::vector<int> id(C, -1);
  int next = 0;
  for (int i = 0; i < C; ++i)
    if (amin[root[i]] == i) id[i] = next++;
  agg.resize(C);
  for (int i = 0; i < C; ++i) agg[i] = id[amin[root[i]]];
  return next;
}

int aggregate(const Bsr& A, const or_config& cfg, std::vector<int32_t>& agg) {
  int nagg = match_pass(A, cfg, agg);
  Bsr G;
  const Bsr* cur = &A;
  std::vector<int32_t> cur_agg = agg;
  for (int pass = 1; pass < cfg.agg_passes; ++pass) {
    Bsr Abar;
    galerkin_tentative(*cur, cur_agg, nagg, Abar);
    std::vector<int32_t> a2;
    int n2 = match_pass(Abar, cfg, a2);
    for (int i = 0; i < A.rows; ++i) agg[i] = a2[agg[i]];
    cur_agg = a2;
    bool stalled = (n2 == nagg);
    nagg = n2;
    G = std::move(Abar);
    cur = &G;
    if (stalled) break;
  }
  return nagg;
}

// Damped block-Jacobi inverse of each diagonal block (same Gauss-Jordan).
int diag_inverses(const Bsr& A, std::vector<double>& dinv) {
  const int n = A.n, nn = n * n;
  dinv.assign((size_t)A.rows * nn, 0.0);
  for (int i = 0; i < A.rows; ++i) {
    int k = find_in_row(A, i, i);
    if (k < 0) return 1;
    if (or_dense_inverse(n, A.blk(k), dinv.data() + (size_t)i * nn)) return 1;
  }
  return 0;
}

// ---- multicolour block DILU (see oracle.h) ----
uint32_t lowbias32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

constexpr int MAX_COLOURS = 128;

// (h(i), i) > (h(j), j)
bool beats(int i, int j) {
  const uint32_t hi = lowbias32((uint32_t)i), hj = lowbias32((uint32_t)j);
  return hi != hj ? hi > hj : i > j;
}

int colour_rows(const Bsr& A, std::vector<int32_t>& colour) {
  const int rows = A.rows;
  colour.assign(rows, -1);
  int left = rows, ncol = 0;
  while (left > 0) {
    // the round's independent set, judged on the state at the round's start
    std::vector<int> pick;
    for (int i = 0; i < rows; ++i) {
      if (colour[i] >= 0) continue;
      bool top = true;
      for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
        const int j = A.ci[k];
        if (j != i && colour[j] < 0 && beats(j, i)) top = false;
      }
      if (top) pick.push_back(i);
    }
    std::vector<int32_t> chosen(pick.size());
    for (size_t q = 0; q < pick.size(); ++q) {
      const int i = pick[q];
      std::vector<bool> used(MAX_COLOURS, false);
      for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
        const int j = A.ci[k];
        if (j != i && colour[j] >= 0) used[colour[j]] = true;
      }
      int c = 0;
      while (c < MAX_COLOURS && used[c]) ++c;
      if (c == MAX_COLOURS) return -1;
      chosen[q] = c;
    }
    for (size_t q = 0; q < pick.size(); ++q) {
      colour[pick[q]] = chosen[q];
      if (chosen[q] + 1 > ncol) ncol = chosen[q] + 1;
    }
    left -= (int)pick.size();
  }
  return ncol;
}

int dilu_factor(const Bsr& A, const std::vector<int32_t>& colour, std::vector<double>& einv) {
  const int n = A.n, nn = n * n, rows = A.rows;
  einv.assign((size_t)rows * nn, 0.0);
  int ncol = 0;
  for (int i = 0; i < rows; ++i) ncol = std::max(ncol, colour[i] + 1);
  std::vector<double> E(nn), W(nn), Z(nn);
  for (int c = 0; c < ncol; ++c)
    for (int i = 0; i < rows; ++i) {
      if (colour[i] != c) continue;
      const int kd = find_in_row(A, i, i);
      if (kd < 0) return 1;
      std::copy(A.blk(kd), A.blk(kd) + nn, E.begin());
      for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
        const int j = A.ci[k];
        if (colour[j] >= c) continue;
        const int kt = find_in_row(A, j, i);
        block_mul(n, A.blk(k), einv.data() + (size_t)j * nn, W.data());
        block_mul(n, W.data(), A.blk(kt), Z.data());
        for (int e = 0; e < nn; ++e) E[e] = E[e] - Z[e];
      }
      if (or_dense_inverse(n, E.data(), einv.data() + (size_t)i * nn)) return 1;
    }
  return 0;
}

// z = M^{-1} r (plain sums, row-major block order)
void dilu_apply(const Bsr& A, const std::vector<int32_t>& colour, int ncol, const std::vector<double>& einv,
                const double* r, double* z) {
  const int n = A.n, nn = n * n, rows = A.rows;
  std::vector<double> y((size_t)rows * n, 0.0), t(n);
  for (int c = 0; c < ncol; ++c)
    for (int i = 0; i < rows; ++i) {
      if (colour[i] != c) continue;
      for (int a = 0; a < n; ++a) t[a] = r[(size_t)i * n + a];
      for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
        const int j = A.ci[k];
        if (colour[j] >= c) continue;
        for (int a = 0; a < n; ++a) {
          double s = 0.0;
          for (int b = 0; b < n; ++b) s += A.blk(k)[a * n + b] * y[(size_t)j * n + b];
          t[a] = t[a] - s;
        }
      }
      for (int a = 0; a < n; ++a) {
        double s = 0.0;
        for (int b = 0; b < n; ++b) s += einv[(size_t)i * nn + a * n + b] * t[b];
        y[(size_t)i * n + a] = s;
      }
    }
  for (int c = ncol - 1; c >= 0; --c)
    for (int i = 0; i < rows; ++i) {
      if (colour[i] != c) continue;
      for (int a = 0; a < n; ++a) t[a] = 0.0;
      for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
        const int j = A.ci[k];
        if (colour[j] <= c) continue;
        for (int a = 0; a < n; ++a) {
          double s = 0.0;
          for (int b = 0; b < n; ++b) s += A.blk(k)[a * n + b] * z[(size_t)j * n + b];
          t[a] = t[a] + s;
        }
      }
      for (int a = 0; a < n; ++a) {
        double s = 0.0;
        for (int b = 0; b < n; ++b) s += einv[(size_t)i * nn + a * n + b] * t[b];
        z[(size_t)i * n + a] = y[(size_t)i * n + a] - s;
      }
    }
}

Bsr bsr_view(int rows, int n, const int32_t* rp, const int32_t* ci, const double* val) {
  Bsr A;
  A.rows = A.cols = rows;
  A.n = n;
  A.rp.assign(rp, rp + rows + 1);
  A.ci.assign(ci, ci + rp[rows]);
  if (val) A.v.assign(val, val + (size_t)rp[rows] * n * n);
  return A;
}

// Smoothed prolongation P = (I - omega_P D^{-1} A) P_tent with
// omega_P = p_omega / rho, rho = max_i sum_j ||D_i^{-1} A_ij||_inf.
// Row i's columns are the sorted aggregates of its neighbours; block
// P_iJ = fma(-omega_P, D_i^{-1} S_iJ, delta) where S_iJ is the sum (row order)
// of A_ij over neighbours j in aggregate J.
void smoothed_P(const Bsr& A, const std::vector<double>& dinv, const std::vector<int32_t>& agg,
                int nagg, double p_omega, Bsr& P, double& omega) {
  const int n = A.n, nn = n * n;
  std::vector<double> T(nn), S(nn);
  double rho = 0.0;
  for (int i = 0; i < A.rows; ++i) {
    double s = 0.0;
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      block_mul(n, dinv.data() + (size_t)i * nn, A.blk(k), T.data());
      double mx = 0.0;
      for (int r = 0; r < n; ++r) {
        double rs = 0.0;
        for (int c = 0; c < n; ++c) rs = rs + std::fabs(T[r * n + c]);
        if (rs > mx) mx = rs;
      }
      s = s + mx;
    }
    if (s > rho) rho = s;
  }
  omega = p_omega / rho;
  P.rows = A.rows;
  P.cols = nagg;
  P.n = n;
  P.rp.assign(A.rows + 1, 0);
  P.ci.clear();
  P.v.clear();
  for (int i = 0; i < A.rows; ++i) {
    std::vector<int> cols;
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) cols.push_back(agg[A.ci[k]]);
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    for (int J : cols) {
      std::fill(S.begin(), S.end(), 0.0);
      for (int k = A.rp[i]; k < A.rp[i + 1]; ++k)
        if (agg[A.ci[k]] == J)
          for (int e = 0; e < nn; ++e) S[e] = S[e] + A.blk(k)[e];
      block_mul(n, dinv.data() + (size_t)i * nn, S.data(), T.data());
      P.ci.push_back(J);
      for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
          double delta = (J == agg[i] && r == c) ? 1.0 : 0.0;
          P.v.push_back(std::fma(-omega, T[r * n + c], delta));
        }
    }
    P.rp[i + 1] = (int32_t)P.ci.size();
  }
}

}  // namespace

struct or_amg {
  struct Level {
    Bsr A;
    std::vector<double> dinv;
    std::vector<int32_t> agg;
    int nagg = 0;
    double omega_p = 0.0;
    Bsr P, R, AP;
    int coarse_kind = -1;  // -1 not coarsest, 0 dense inverse, 1 sweeps
    // multicolour DILU (smoother = 1); ncol = -1: this level keeps block Jacobi
    std::vector<int32_t> colour;
    int ncol = -1;
    std::vector<double> einv;
  };
  int n = 0;
  or_config cfg{};
  std::vector<Level> lv;
  std::vector<double> cinv;
};

namespace {

int finish_coarsest(or_amg* h, int l) {
  auto& L = h->lv[l];
  const int N = L.A.rows * h->n;
  if (N <= h->cfg.coarse_dense_max) {
    std::vector<double> M((size_t)N * N, 0.0);
    const int n = h->n;
    for (int i = 0; i < L.A.rows; ++i)
      for (int k = L.A.rp[i]; k < L.A.rp[i + 1]; ++k)
        for (int r = 0; r < n; ++r)
          for (int c = 0; c < n; ++c)
            M[(size_t)(i * n + r) * N + L.A.ci[k] * n + c] = L.A.blk(k)[r * n + c];
    h->cinv.assign((size_t)N * N, 0.0);
    if (or_dense_inverse(N, M.data(), h->cinv.data())) return 6;
    L.coarse_kind = 0;
  } else {
    L.coarse_kind = 1;
  }
  return 0;
}

// Transfer operators and coarse matrix for level l (aggregates already set).
void build_transfer(or_amg* h, int l) {
  auto& L = h->lv[l];
  if (h->cfg.pmode == 1) {
    L.P = tentative_P(L.A.rows, h->n, L.agg, L.nagg);
    L.omega_p = 0.0;
  } else {
    smoothed_P(L.A, L.dinv, L.agg, L.nagg, h->cfg.p_omega, L.P, L.omega_p);
  }
  Bsr Ac;
  if (h->cfg.pmode == 1) {
    transpose(L.P, L.R);
    galerkin_tentative(L.A, L.agg, L.nagg, Ac);
  } else {
    galerkin(L.A, L.P, L.R, L.AP, Ac);
  }
  if ((int)h->lv.size() <= l + 1) h->lv.emplace_back();
  h->lv[l + 1].A = std::move(Ac);
}

}  // namespace

extern "C" {

or_amg* or_amg_setup(int rows, int n, const int32_t* rp, const int32_t* ci, const double* val,
                     const or_config* cfg, int* status) {
  or_amg* h = new or_amg();
  h->n = n;
  h->cfg = *cfg;
  h->lv.emplace_back();
  Bsr& A0 = h->lv[0].A;
  A0.rows = rows;
  A0.cols = rows;
  A0.n = n;
  A0.rp.assign(rp, rp + rows + 1);
  A0.ci.assign(ci, ci + rp[rows]);
  A0.v.assign(val, val + (size_t)rp[rows] * n * n);
  *status = 0;
  for (int l = 0;; ++l) {
    auto& L = h->lv[l];
    if (diag_inverses(L.A, L.dinv)) { *status = 6; return h; }
    if (cfg->smoother == 1) {
      L.ncol = colour_rows(L.A, L.colour);
      if (L.ncol > 0 && dilu_factor(L.A, L.colour, L.einv)) { *status = 6; return h; }
    } else if (cfg->smoother == 2) {
      // SGS: the DILU form with E = D (no modification of the diagonal)
      L.ncol = colour_rows(L.A, L.colour);
      if (L.ncol > 0) L.einv = L.dinv;
    }
    const int C = L.A.rows;
    bool last = C <= cfg->coarse_size || l == cfg->max_levels - 1;
    if (!last) {
      L.nagg = aggregate(L.A, *cfg, L.agg);
      if (L.nagg >= C || L.nagg > cfg->max_coarsen_ratio * C) {
        last = true;
        L.agg.clear();
        L.nagg = 0;
      }
    }
    if (last) {
      *status = finish_coarsest(h, l);
      return h;
    }
    build_transfer(h, l);
  }
}

int or_amg_resetup(or_amg* h, const double* val) {
  auto& A0 = h->lv[0].A;
  A0.v.assign(val, val + (size_t)A0.nnz() * h->n * h->n);
  const int L = (int)h->lv.size();
  for (int l = 0; l < L; ++l) {
    auto& lev = h->lv[l];
    if (diag_inverses(lev.A, lev.dinv)) return 6;
    if (lev.ncol > 0 && dilu_factor(lev.A, lev.colour, lev.einv)) return 6;
    if (lev.coarse_kind >= 0) return finish_coarsest(h, l);
    build_transfer(h, l);
  }
  return 0;
}

void or_amg_free(or_amg* h) { delete h; }
int or_amg_levels(const or_amg* h) { return (int)h->lv.size(); }

void or_amg_level_info(const or_amg* h, int l, int* rows, int* nnz, int* p_nnz, int* kind) {
  const auto& L = h->lv[l];
  *rows = L.A.rows;
  *nnz = L.A.nnz();
  *p_nnz = L.coarse_kind >= 0 ? 0 : L.P.nnz();
  *kind = L.coarse_kind;
}

void or_amg_get_A(const or_amg* h, int l, int32_t* rp, int32_t* ci, double* val) {
  const auto& A = h->lv[l].A;
  if (rp) std::copy(A.rp.begin(), A.rp.end(), rp);
  if (ci) std::copy(A.ci.begin(), A.ci.end(), ci);
  if (val) std::copy(A.v.begin(), A.v.end(), val);
}

void or_amg_get_P(const or_amg* h, int l, int32_t* rp, int32_t* ci, double* val, int32_t* agg,
                  double* omega) {
  const auto& L = h->lv[l];
  if (rp) std::copy(L.P.rp.begin(), L.P.rp.end(), rp);
  if (ci) std::copy(L.P.ci.begin(), L.P.ci.end(), ci);
  if (val) std::copy(L.P.v.begin(), L.P.v.end(), val);
  if (agg) std::copy(L.agg.begin(), L.agg.end(), agg);
  if (omega) *omega = L.omega_p;
}

void or_amg_get_dinv(const or_amg* h, int l, double* dinv) {
  std::copy(h->lv[l].dinv.begin(), h->lv[l].dinv.end(), dinv);
}

int or_amg_get_dilu(const or_amg* h, int l, int32_t* colour, double* einv) {
  const auto& L = h->lv[l];
  if (L.ncol <= 0) return -1;
  if (colour) std::copy(L.colour.begin(), L.colour.end(), colour);
  if (einv) std::copy(L.einv.begin(), L.einv.end(), einv);
  return L.ncol;
}

int or_colour(int rows, const int32_t* rp, const int32_t* ci, int32_t* colour) {
  Bsr A = bsr_view(rows, 1, rp, ci, nullptr);
  std::vector<int32_t> c;
  const int nc = colour_rows(A, c);
  std::copy(c.begin(), c.end(), colour);
  return nc;
}

int or_dilu_factor(int rows, int n, const int32_t* rp, const int32_t* ci, const double* val,
                   const int32_t* colour, double* einv) {
  Bsr A = bsr_view(rows, n, rp, ci, val);
  std::vector<int32_t> c(colour, colour + rows);
  std::vector<double> e;
  const int st = dilu_factor(A, c, e);
  std::copy(e.begin(), e.end(), einv);
  return st;
}

void or_dilu_apply(int rows, int n, const int32_t* rp, const int32_t* ci, const double* val,
                   const int32_t* colour, int ncolours, const double* einv, const double* r, double* z) {
  Bsr A = bsr_view(rows, n, rp, ci, val);
  std::vector<int32_t> c(colour, colour + rows);
  std::vector<double> e(einv, einv + (size_t)rows * n * n);
  dilu_apply(A, c, ncolours, e, r, z);
}

void or_amg_get_coarse_inverse(const or_amg* h, double* inv) {
  std::copy(h->cinv.begin(), h->cinv.end(), inv);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// V-cycle (preconditioner). Reading: damped block Jacobi
//   x <- x + omega D^{-1} (b - A x), nu1 sweeps before and nu2 after, the first
//   pre-sweep from x = 0 being x = omega D^{-1} b; restriction R = P^T;
//   coarsest level: dense inverse, or coarse_sweeps sweeps when too large.
// ---------------------------------------------------------------------------
namespace {

void jacobi_sweep(const Bsr& A, const std::vector<double>& dinv, double omega, const double* b,
                  std::vector<double>& x) {
  const int n = A.n, nn = n * n;
  std::vector<double> r((size_t)A.rows * n);
  or_bsr_spmv(A.rows, n, A.rp.data(), A.ci.data(), A.v.data(), x.data(), r.data());
#pragma omp parallel for schedule(static)
  for (size_t e = 0; e < r.size(); ++e) r[e] = b[e] - r[e];
#pragma omp parallel for schedule(static)
  for (int i = 0; i < A.rows; ++i)
    for (int a = 0; a < n; ++a) {
      double t = 0.0;
      for (int c = 0; c < n; ++c) t += dinv[(size_t)i * nn + a * n + c] * r[(size_t)i * n + c];
      x[(size_t)i * n + a] = x[(size_t)i * n + a] + omega * t;
    }
}

// DILU step x <- x + M^{-1} (b - A x)
void dilu_sweep(const Bsr& A, const std::vector<int32_t>& colour, int ncol, const std::vector<double>& einv,
                const double* b, std::vector<double>& x) {
  const size_t N = (size_t)A.rows * A.n;
  std::vector<double> r(N), d(N);
  or_bsr_spmv(A.rows, A.n, A.rp.data(), A.ci.data(), A.v.data(), x.data(), r.data());
  for (size_t e = 0; e < N; ++e) r[e] = b[e] - r[e];
  dilu_apply(A, colour, ncol, einv, r.data(), d.data());
  for (size_t e = 0; e < N; ++e) x[e] = x[e] + d[e];
}

void vcycle(const or_amg* h, int l, const double* b, std::vector<double>& x);

// One smoothing step on level l with the configured smoother.
void smooth(const or_amg* h, int l, const double* b, std::vector<double>& x) {
  const auto& L = h->lv[l];
  if (L.ncol > 0) dilu_sweep(L.A, L.colour, L.ncol, L.einv, b, x);
  else jacobi_sweep(L.A, L.dinv, h->cfg.jacobi_omega, b, x);
}

void vcycle(const or_amg* h, int l, const double* b, std::vector<double>& x) {
  const auto& L = h->lv[l];
  const int n = h->n, nn = n * n, N = L.A.rows * n;
  const double om = h->cfg.jacobi_omega;
  x.assign(N, 0.0);
  if (L.ncol > 0 && L.coarse_kind != 0) {
    // DILU: every sweep, the first one included, is the general step from x
    if (L.coarse_kind == 1) {
      for (int s = 0; s < h->cfg.coarse_sweeps; ++s) smooth(h, l, b, x);
      return;
    }
    for (int s = 0; s < h->cfg.nu1; ++s) smooth(h, l, b, x);
    std::vector<double> r(N), bc((size_t)L.P.cols * n), xc;
    or_bsr_spmv(L.A.rows, n, L.A.rp.data(), L.A.ci.data(), L.A.v.data(), x.data(), r.data());
    for (int e = 0; e < N; ++e) r[e] = b[e] - r[e];
    or_bsr_spmv(L.R.rows, n, L.R.rp.data(), L.R.ci.data(), L.R.v.data(), r.data(), bc.data());
    vcycle(h, l + 1, bc.data(), xc);
    std::vector<double> px(N);
    or_bsr_spmv(L.P.rows, n, L.P.rp.data(), L.P.ci.data(), L.P.v.data(), xc.data(), px.data());
    for (int e = 0; e < N; ++e) x[e] = x[e] + px[e];
    for (int s = 0; s < h->cfg.nu2; ++s) smooth(h, l, b, x);
    return;
  }
  if (L.coarse_kind == 0) {
#pragma omp parallel for schedule(static)
    for (int r = 0; r < N; ++r) {
      double t = 0.0;
      for (int c = 0; c < N; ++c) t += h->cinv[(size_t)r * N + c] * b[c];
      x[r] = t;
    }
    return;
  }
  if (L.coarse_kind == 1) {
    for (int s = 0; s < h->cfg.coarse_sweeps; ++s) jacobi_sweep(L.A, L.dinv, om, b, x);
    return;
  }
  if (h->cfg.nu1 >= 1) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < L.A.rows; ++i)
      for (int a = 0; a < n; ++a) {
        double t = 0.0;
        for (int c = 0; c < n; ++c) t += L.dinv[(size_t)i * nn + a * n + c] * b[(size_t)i * n + c];
        x[(size_t)i * n + a] = om * t;
      }
    for (int s = 1; s < h->cfg.nu1; ++s) jacobi_sweep(L.A, L.dinv, om, b, x);
  }
  std::vector<double> r(N), bc((size_t)L.P.cols * n), xc;
  or_bsr_spmv(L.A.rows, n, L.A.rp.data(), L.A.ci.data(), L.A.v.data(), x.data(), r.data());
#pragma omp parallel for schedule(static)
  for (int e = 0; e < N; ++e) r[e] = b[e] - r[e];
  or_bsr_spmv(L.R.rows, n, L.R.rp.data(), L.R.ci.data(), L.R.v.data(), r.data(), bc.data());
  vcycle(h, l + 1, bc.data(), xc);
  std::vector<double> px(N);
  or_bsr_spmv(L.P.rows, n, L.P.rp.data(), L.P.ci.data(), L.P.v.data(), xc.data(), px.data());
#pragma omp parallel for schedule(static)
  for (int e = 0; e < N; ++e) x[e] = x[e] + px[e];
  for (int s = 0; s < h->cfg.nu2; ++s) jacobi_sweep(L.A, L.dinv, om, b, x);
}

}  // namespace

extern "C" void or_amg_vcycle(const or_amg* h, const double* v, double* z) {
  std::vector<double> x;
  vcycle(h, 0, v, x);
  std::copy(x.begin(), x.end(), z);
}

// ---------------------------------------------------------------------------
// Krylov solvers. FGMRES(m): right-preconditioned flexible GMRES (GMRES of
// Saad & Schultz, Sec. 2; flexible because the preconditioner may vary),
// classical Gram-Schmidt applied twice, Givens rotations, restart after m
// steps. Stopping reading: the rotated residual |g_{j+1}| / ||b|| <= tol ends a
// cycle; convergence is decided on the true residual ||b - A x|| / ||b||
// recomputed at the end of every cycle. Happy breakdown when
// h_{j+1,j} <= 1e-14 ||A z_j||.
// BiCGStab (van der Vorst), right-preconditioned, with r_hat = r_0; a
// converged recurrence residual is confirmed with the true residual, and
// restarted from it if the check fails; rho = 0, (r_hat, v) = 0 or
// (t, t) = 0 restart once from the true residual, then report breakdown.
// ---------------------------------------------------------------------------
namespace {

struct Sys {
  int rows, n, N;
  const int32_t *rp, *ci;
  const double* val;
  const or_amg* h;
  const or_config* cfg;
  std::vector<double> dinv;
  // precond = 3: multicolour block SGS, M = (D + L) D^-1 (D + U) with the
  // colour order of the DILU smoother (ncol <= 0: more colours than allowed,
  // block Jacobi instead)
  Bsr A;
  std::vector<int32_t> colour;
  int ncol = 0;
};

double dot(const std::vector<double>& a, const std::vector<double>& b) {
  double s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}
double nrm2(const std::vector<double>& a) { return std::sqrt(dot(a, a)); }

void matvec(const Sys& S, const std::vector<double>& x, std::vector<double>& y) {
  y.resize(S.N);
  or_bsr_spmv(S.rows, S.n, S.rp, S.ci, S.val, x.data(), y.data());
}

void precond(const Sys& S, const std::vector<double>& v, std::vector<double>& z) {
  z.resize(S.N);
  if (S.cfg->precond == 0) {
    or_amg_vcycle(S.h, v.data(), z.data());
  } else if (S.cfg->precond == 3 && S.ncol > 0) {
    dilu_apply(S.A, S.colour, S.ncol, S.dinv, v.data(), z.data());
  } else if (S.cfg->precond == 2 || S.cfg->precond == 3) {
    const int n = S.n, nn = n * n;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < S.rows; ++i)
      for (int a = 0; a < n; ++a) {
        double t = 0.0;
        for (int c = 0; c < n; ++c) t += S.dinv[(size_t)i * nn + a * n + c] * v[(size_t)i * n + c];
        z[(size_t)i * n + a] = t;
      }
  } else {
    z = v;
  }
}

void true_residual(const Sys& S, const double* b, const std::vector<double>& x,
                   std::vector<double>& r) {
  matvec(S, x, r);
#pragma omp parallel for schedule(static)
  for (int e = 0; e < S.N; ++e) r[e] = b[e] - r[e];
}

// One Arnoldi step of FGMRES: returns h (j+2 entries) and the new vector.
// Returns 1 on happy breakdown.
int arnoldi_step(const Sys& S, std::vector<std::vector<double>>& V,
                 std::vector<std::vector<double>>& Z, int j, std::vector<double>& h) {
  precond(S, V[j], Z[j]);
  std::vector<double> w;
  matvec(S, Z[j], w);
  const double wn0 = nrm2(w);
  h.assign(j + 2, 0.0);
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<double> c(j + 1);
    for (int i = 0; i <= j; ++i) c[i] = dot(V[i], w);
#pragma omp parallel for schedule(static)
    for (int e = 0; e < S.N; ++e) {
      double t = w[e];
      for (int i = 0; i <= j; ++i) t -= c[i] * V[i][e];
      w[e] = t;
    }
    for (int i = 0; i <= j; ++i) h[i] += c[i];
  }
  const double hn = nrm2(w);
  h[j + 1] = hn;
  if (!(hn > 1e-14 * wn0)) return 1;
  V[j + 1].resize(S.N);
#pragma omp parallel for schedule(static)
  for (int e = 0; e < S.N; ++e) V[j + 1][e] = w[e] / hn;
  return 0;
}

int fgmres(const Sys& S, const double* b, double* x0, or_result* res, double* hist, int hist_len) {
  const int N = S.N, m = S.cfg->restart;
  std::vector<double> bb(b, b + N), x(x0, x0 + N), r;
  const double bnorm = nrm2(bb);
  res->iters = 0;
  res->restarts = 0;
  if (bnorm == 0.0) {
    std::fill(x0, x0 + N, 0.0);
    res->rel_res_initial = res->rel_res_final = 0.0;
    return 0;
  }
  true_residual(S, b, x, r);
  double beta = nrm2(r);
  res->rel_res_initial = beta / bnorm;
  res->rel_res_final = beta / bnorm;
  if (beta <= S.cfg->tol * bnorm) return 0;
  int iters = 0, status = 0;
  std::vector<std::vector<double>> V(m + 1), Z(m);
  std::vector<double> H((size_t)(m + 1) * m, 0.0), g(m + 1), cs(m), sn(m), h;
  for (;;) {
    V[0].resize(N);
#pragma omp parallel for schedule(static)
    for (int e = 0; e < N; ++e) V[0][e] = r[e] / beta;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jend = 0;
    for (int j = 0; j < m; ++j) {
      int happy = arnoldi_step(S, V, Z, j, h);
      for (int i = 0; i <= j + 1; ++i) H[(size_t)i * m + j] = h[i];
      for (int i = 0; i < j; ++i) {
        double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
      if (c == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
      else {
        double d = std::sqrt(a * a + c * c);
        cs[j] = a / d;
        sn[j] = c / d;
      }
      H[(size_t)j * m + j] = cs[j] * a + sn[j] * c;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++iters;
      jend = j + 1;
      if (hist && iters <= hist_len) hist[iters - 1] = std::fabs(g[j + 1]) / bnorm;
      if (happy) break;
      if (std::fabs(g[j + 1]) <= S.cfg->tol * bnorm || iters >= S.cfg->maxiter) break;
    }
    std::vector<double> y(jend);
    for (int i = jend - 1; i >= 0; --i) {
      double t = g[i];
      for (int k = i + 1; k < jend; ++k) t -= H[(size_t)i * m + k] * y[k];
      y[i] = t / H[(size_t)i * m + i];
    }
#pragma omp parallel for schedule(static)
    for (int e = 0; e < N; ++e) {
      double t = x[e];
      for (int j = 0; j < jend; ++j) t += y[j] * Z[j][e];
      x[e] = t;
    }
    true_residual(S, b, x, r);
    beta = nrm2(r);
    res->rel_res_final = beta / bnorm;
    if (beta <= S.cfg->tol * bnorm) { status = 0; break; }
    if (!std::isfinite(beta)) { status = 5; break; }
    if (iters >= S.cfg->maxiter) { status = 4; break; }
    res->restarts++;
  }
  res->iters = iters;
  std::copy(x.begin(), x.end(), x0);
  return status;
}

// Per-iteration record of BiCGStab's iterate x_k and its recurrence residual
// (the vector the recurrence carries as b - A x_k: r_k after a full step, s
// after a half step that ends the solve). Test hook.
struct Trace {
  double* x = nullptr;
  double* r = nullptr;
  int cap = 0;
  int count = 0;
  void record(const std::vector<double>& xv, const std::vector<double>& rv) {
    if (count >= cap) return;
    const size_t N = xv.size();
    std::copy(xv.begin(), xv.end(), x + (size_t)count * N);
    std::copy(rv.begin(), rv.end(), r + (size_t)count * N);
    ++count;
  }
};

int bicgstab(const Sys& S, const double* b, double* x0, or_result* res, double* hist, int hist_len,
             Trace* tr) {
  const int N = S.N;
  const double tol = S.cfg->tol;
  std::vector<double> bb(b, b + N), x(x0, x0 + N), r, rhat, p(N, 0.0), v(N, 0.0), s(N), t, ph, sh;
  const double bnorm = nrm2(bb);
  res->iters = 0;
  res->restarts = 0;
  if (bnorm == 0.0) {
    std::fill(x0, x0 + N, 0.0);
    res->rel_res_initial = res->rel_res_final = 0.0;
    return 0;
  }
  true_residual(S, b, x, r);
  res->rel_res_initial = res->rel_res_final = nrm2(r) / bnorm;
  if (nrm2(r) <= tol * bnorm) return 0;
  rhat = r;
  double rho_old = 1.0, alpha = 1.0, omega = 1.0;
  bool first = true, restarted = false;
  int status = 4, it = 0;
  auto restart = [&](bool breakdown) -> bool {
    if (breakdown) {
      if (restarted) return false;
      restarted = true;
    }
    true_residual(S, b, x, r);
    rhat = r;
    first = true;
    res->restarts++;
    return true;
  };
  while (it < S.cfg->maxiter) {
    double rho = dot(rhat, r);
    if (rho == 0.0 || !std::isfinite(rho)) {
      if (!restart(true)) { status = 5; break; }
      continue;
    }
    if (first) p = r;
    else {
      double beta = (rho / rho_old) * (alpha / omega);
#pragma omp parallel for schedule(static)
      for (int e = 0; e < N; ++e) p[e] = r[e] + beta * (p[e] - omega * v[e]);
    }
    first = false;
    precond(S, p, ph);
    matvec(S, ph, v);
    double den = dot(rhat, v);
    if (den == 0.0 || !std::isfinite(den)) {
      if (!restart(true)) { status = 5; break; }
      continue;
    }
    alpha = rho / den;
#pragma omp parallel for schedule(static)
    for (int e = 0; e < N; ++e) s[e] = r[e] - alpha * v[e];
    ++it;
    double sn = nrm2(s);
    if (sn <= tol * bnorm) {
      for (int e = 0; e < N; ++e) x[e] = x[e] + alpha * ph[e];
      if (hist && it <= hist_len) hist[it - 1] = sn / bnorm;
      if (tr) tr->record(x, s);
      true_residual(S, b, x, r);
      if (nrm2(r) <= tol * bnorm) { status = 0; break; }
      restart(false);
      continue;
    }
    precond(S, s, sh);
    matvec(S, sh, t);
    double tt = dot(t, t);
    if (tt == 0.0 || !std::isfinite(tt)) {
      if (!restart(true)) { status = 5; break; }
      continue;
    }
    omega = dot(t, s) / tt;
#pragma omp parallel for schedule(static)
    for (int e = 0; e < N; ++e) {
      x[e] = x[e] + alpha * ph[e] + omega * sh[e];
      r[e] = s[e] - omega * t[e];
    }
    rho_old = rho;
    double rn = nrm2(r);
    if (hist && it <= hist_len) hist[it - 1] = rn / bnorm;
    if (tr) tr->record(x, r);
    if (rn <= tol * bnorm) {
      true_residual(S, b, x, r);
      if (nrm2(r) <= tol * bnorm) { status = 0; break; }
      restart(false);
      continue;
    }
    if (omega == 0.0) {
      if (!restart(true)) { status = 5; break; }
    }
  }
  true_residual(S, b, x, r);
  res->rel_res_final = nrm2(r) / bnorm;
  if (status == 4 && res->rel_res_final <= tol) status = 0;
  res->iters = it;
  std::copy(x.begin(), x.end(), x0);
  return status;
}

Sys make_sys(int rows, int n, const int32_t* rp, const int32_t* ci, const double* val,
             const or_amg* h, const or_config* cfg, int* bad) {
  Sys S{rows, n, rows * n, rp, ci, val, h, cfg, {}, {}, {}, 0};
  *bad = 0;
  if (cfg->precond == 2 || cfg->precond == 3) {
    Bsr& A = S.A;
    A.rows = rows;
    A.cols = rows;
    A.n = n;
    A.rp.assign(rp, rp + rows + 1);
    A.ci.assign(ci, ci + rp[rows]);
    A.v.assign(val, val + (size_t)rp[rows] * n * n);
    *bad = diag_inverses(A, S.dinv);
    if (cfg->precond == 3) S.ncol = colour_rows(A, S.colour);
  }
  return S;
}

}  // namespace

extern "C" int or_solve_trace(int rows, int n, const int32_t* rp, const int32_t* ci, const double* val,
                              const or_amg* h, const or_config* cfg, const double* b, double* x,
                              or_result* res, double* hist, int hist_len, double* xtrace, double* rtrace,
                              int trace_len) {
  int bad = 0;
  Sys S = make_sys(rows, n, rp, ci, val, h, cfg, &bad);
  res->levels = h ? or_amg_levels(h) : 0;
  if (bad) { res->status = 6; return 6; }
  Trace tr;
  tr.x = xtrace;
  tr.r = rtrace;
  tr.cap = (xtrace && rtrace) ? trace_len : 0;
  int st = cfg->solver == 1 ? bicgstab(S, b, x, res, hist, hist_len, tr.cap > 0 ? &tr : nullptr)
                            : fgmres(S, b, x, res, hist, hist_len);
  res->status = st;
  return tr.cap > 0 ? tr.count : st;
}

extern "C" int or_solve(int rows, int n, const int32_t* rp, const int32_t* ci, const double* val,
                        const or_amg* h, const or_config* cfg, const double* b, double* x,
                        or_result* res, double* hist, int hist_len) {
  return or_solve_trace(rows, n, rp, ci, val, h, cfg, b, x, res, hist, hist_len, nullptr, nullptr, 0);
}

extern "C" int or_fgmres_arnoldi(int rows, int n, const int32_t* rp, const int32_t* ci,
                                 const double* val, const or_amg* h, const or_config* cfg,
                                 const double* b, int jsteps, double* Vout, double* Zout,
                                 double* Hout) {
  int bad = 0;
  Sys S = make_sys(rows, n, rp, ci, val, h, cfg, &bad);
  if (bad) return 6;
  const int N = S.N;
  std::vector<double> bb(b, b + N);
  const double beta = nrm2(bb);
  std::vector<std::vector<double>> V(jsteps + 1), Z(jsteps);
  V[0].resize(N);
  for (int e = 0; e < N; ++e) V[0][e] = b[e] / beta;
  std::vector<double> h_;
  int done = 0;
  for (int j = 0; j < jsteps; ++j) {
    int happy = arnoldi_step(S, V, Z, j, h_);
    for (int i = 0; i <= j + 1; ++i) Hout[(size_t)i * jsteps + j] = h_[i];
    done = j + 1;
    if (happy) break;
  }
  for (int j = 0; j <= done && j <= jsteps; ++j)
    if (!V[j].empty()) std::copy(V[j].begin(), V[j].end(), Vout + (size_t)j * N);
  for (int j = 0; j < done; ++j) std::copy(Z[j].begin(), Z[j].end(), Zout + (size_t)j * N);
  return done;
}

extern "C" int or_aggregate(int rows, int n, const int32_t* rp, const int32_t* ci,
                            const double* val, const or_config* cfg, int32_t* agg_out) {
  Bsr A;
  A.rows = rows;
  A.cols = rows;
  A.n = n;
  A.rp.assign(rp, rp + rows + 1);
  A.ci.assign(ci, ci + rp[rows]);
  A.v.assign(val, val + (size_t)rp[rows] * n * n);
  std::vector<int32_t> agg;
  int na = aggregate(A, *cfg, agg);
  std::copy(agg.begin(), agg.end(), agg_out);
  return na;
}
