"""Oracle pins for the AMG setup and V-cycle (Sec. 2.3: aggregation AMG for
block-coupled systems; the rule itself is a documented reading).

Pinned against: numpy/LAPACK inverses, hand-worked aggregation cases
(golden), partition / connectivity / numbering invariants, dense Galerkin
triple products, the 1-D Laplacian's closed-form prolongation weight, the
two-grid error-propagation operator, linearity and symmetry of the cycle.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2403_07882_b300 import synth
from test_oracle_format import dense_from_bsr

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def scalar_chain(diag, couplings):
    C = len(diag)
    owner = np.array([c[0] for c in couplings], np.int32)
    nb = np.array([c[1] for c in couplings], np.int32)
    val = np.array([c[2] for c in couplings])
    sys = dict(n_cells=C, n_faces=len(couplings), n=1, owner=owner, neighbour=nb,
               diag=np.array(diag, float).reshape(C, 1, 1), upper=val.reshape(-1, 1, 1).copy(),
               lower=val.reshape(-1, 1, 1).copy())
    return oracle.ldu_to_bsr(sys)


# ---------------------------------------------------------------- inverses
def test_dense_inverse_vs_lapack():
    rng = np.random.default_rng(0)
    for N in (1, 2, 5, 17, 40):
        A = rng.standard_normal((N, N)) + N * np.eye(N)
        inv = oracle.dense_inverse(A)
        assert np.allclose(inv, np.linalg.inv(A), rtol=1e-12, atol=1e-13)
        assert np.allclose(A @ inv, np.eye(N), atol=1e-12)


def test_dense_inverse_needs_pivoting():
    A = np.array([[0.0, 2.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 4.0]])
    inv = oracle.dense_inverse(A)
    assert np.array_equal(inv, np.array([[0.0, 1.0, 0.0], [0.5, 0.0, 0.0], [0.0, 0.0, 0.25]]))


def test_dense_inverse_permutation_exact():
    P = np.eye(6)[[3, 0, 5, 1, 2, 4]]
    assert np.array_equal(oracle.dense_inverse(P), P.T)


def test_dense_inverse_singular():
    with pytest.raises(np.linalg.LinAlgError):
        oracle.dense_inverse(np.array([[1.0, 2.0], [2.0, 4.0]]))


# ------------------------------------------------------------ aggregation
@pytest.mark.parametrize("case", ["case_distinct", "case_pairs", "case_tie", "case_leftover_min"])
def test_aggregation_golden(case):
    g = json.load(open(os.path.join(GOLD, "aggregation_chain4.json")))[case]
    bsr = scalar_chain(g["diag"], g["couplings"])
    agg, na = oracle.aggregate(bsr, oracle.config(agg_passes=1))
    assert agg.tolist() == g["agg_one_pass"] and na == g["nagg_one_pass"]


def check_partition(bsr, agg, na):
    assert agg.min() == 0 and agg.max() == na - 1
    assert len(np.unique(agg)) == na
    # canonical numbering: ids ascend with each aggregate's smallest member
    first = np.array([np.flatnonzero(agg == a)[0] for a in range(na)])
    assert np.all(np.diff(first) > 0)
    # every aggregate is connected in the matrix graph
    rp, col = bsr["row_ptr"], bsr["col"]
    for a in range(na):
        members = set(np.flatnonzero(agg == a).tolist())
        seen, stack = set(), [min(members)]
        while stack:
            i = stack.pop()
            if i in seen:
                continue
            seen.add(i)
            stack.extend(j for j in col[rp[i]:rp[i + 1]] if j in members and j not in seen)
        assert seen == members


@pytest.mark.parametrize("gen", [lambda: synth.density(8, seed=1), lambda: synth.pressure(6, seed=2),
                                 lambda: synth.random_graph(60, 150, 3, seed=4)])
def test_aggregation_invariants(gen):
    sys = gen()
    bsr = oracle.ldu_to_bsr(sys)
    for passes in (1, 2):
        agg, na = oracle.aggregate(bsr, oracle.config(agg_passes=passes))
        check_partition(bsr, agg, na)
        assert na < bsr["rows"]
        agg2, na2 = oracle.aggregate(bsr, oracle.config(agg_passes=passes))
        assert np.array_equal(agg, agg2) and na == na2


def test_aggregation_invariant_under_block_permutation():
    """Frobenius norms, hence aggregates, ignore a symmetric permutation of
    the unknowns inside every block (e.g. (u, p) vs (p, u) ordering)."""
    sys = synth.pressure(6, seed=3)
    perm = [1, 2, 3, 0]
    alt = dict(sys)
    for key in ("diag", "upper", "lower"):
        alt[key] = np.ascontiguousarray(sys[key][:, perm][:, :, perm])
    a1, n1 = oracle.aggregate(oracle.ldu_to_bsr(sys))
    a2, n2 = oracle.aggregate(oracle.ldu_to_bsr(alt))
    assert n1 == n2 and np.array_equal(a1, a2)


# ------------------------------------------------------ transfer operators
def hierarchy(sys, **kw):
    bsr = oracle.ldu_to_bsr(sys)
    amg = oracle.Amg(bsr, oracle.config(**kw))
    assert amg.status == 0
    return bsr, amg


def ptent_dense(agg, na, n):
    P = np.zeros((agg.size * n, na * n))
    for i, a in enumerate(agg):
        P[i * n:(i + 1) * n, a * n:(a + 1) * n] = np.eye(n)
    return P


@pytest.mark.parametrize("pmode", [0, 1])
def test_galerkin_vs_dense(pmode):
    sys = synth.density(5, 4, 3, seed=9)
    bsr, amg = hierarchy(sys, pmode=pmode, coarse_size=4)
    assert amg.levels >= 3
    for l in range(amg.levels - 1):
        A = dense_from_bsr(amg.A(l))
        P = amg.P(l)
        Pd = dense_from_bsr(P)
        Ac = dense_from_bsr(amg.A(l + 1))
        ref = Pd.T @ A @ Pd
        assert np.allclose(Ac, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
        if pmode == 1:
            assert np.array_equal(Pd, ptent_dense(P["agg"], amg.info(l + 1)["rows"], sys["n"]))


def test_tentative_galerkin_is_block_sums():
    sys = synth.random_graph(40, 90, 2, seed=8)
    bsr, amg = hierarchy(sys, pmode=1, coarse_size=2)
    agg = amg.P(0)["agg"]
    Ac = amg.A(1)
    n = 2
    dense = dense_from_bsr(amg.A(0))
    na = amg.info(1)["rows"]
    for I in range(na):
        for k in range(Ac["row_ptr"][I], Ac["row_ptr"][I + 1]):
            J = Ac["col"][k]
            s = np.zeros((n, n))
            for i in np.flatnonzero(agg == I):
                for j in np.flatnonzero(agg == J):
                    s += dense[i * n:(i + 1) * n, j * n:(j + 1) * n]
            assert np.allclose(Ac["val"][k], s, rtol=1e-14, atol=1e-14)


def test_smoothed_p_dense_formula():
    sys = synth.density(4, 4, 3, seed=12)
    bsr, amg = hierarchy(sys, pmode=0, coarse_size=4)
    n = sys["n"]
    P = amg.P(0)
    A = dense_from_bsr(amg.A(0))
    Dinv = np.zeros_like(A)
    for i, blk in enumerate(amg.dinv(0)):
        Dinv[i * n:(i + 1) * n, i * n:(i + 1) * n] = blk
    T = Dinv @ A
    rho = max(sum(np.abs(T[i * n:(i + 1) * n, j * n:(j + 1) * n]).sum(1).max()
                  for j in range(bsr["rows"])) for i in range(bsr["rows"]))
    assert P["omega"] == pytest.approx(4.0 / 3.0 / rho, rel=1e-14)
    Pt = ptent_dense(P["agg"], amg.info(1)["rows"], n)
    ref = (np.eye(A.shape[0]) - P["omega"] * T) @ Pt
    assert np.allclose(dense_from_bsr(P), ref, rtol=1e-13, atol=1e-14)


def test_smoothed_p_laplacian_closed_form():
    """1-D Laplacian tridiag(-1, 2, -1): sum_j |D^-1 A_ij| = 2 in every
    interior row, so omega_P = (4/3)/2 = 2/3, the classical smoothed-
    aggregation damping; a zero-row-sum operator keeps P's row sums at 1."""
    C = 12
    couplings = [[i, i + 1, -1.0] for i in range(C - 1)]
    diag = [2.0] * C
    bsr = scalar_chain(diag, couplings)
    amg = oracle.Amg(bsr, oracle.config(pmode=0, coarse_size=2, agg_passes=1))
    P = amg.P(0)
    assert P["omega"] == pytest.approx(2.0 / 3.0, rel=1e-15)
    # interior rows (not touching the two boundary cells) sum to exactly 1
    Pd = dense_from_bsr(P)
    sums = Pd.sum(1)
    assert np.allclose(sums[1:-1], 1.0, rtol=0, atol=1e-15)


def test_dinv_vs_lapack():
    sys = synth.pressure(4, seed=5)
    bsr, amg = hierarchy(sys)
    d = amg.dinv(0)
    blocks = bsr["val"][bsr["pos_diag"]]
    assert np.allclose(d, np.linalg.inv(blocks), rtol=1e-12, atol=1e-13)


def test_coarse_inverse_vs_lapack():
    sys = synth.density(6, seed=4)
    bsr, amg = hierarchy(sys)
    L = amg.levels - 1
    assert amg.info(L)["coarse_kind"] == 0
    A = dense_from_bsr(amg.A(L))
    assert np.allclose(amg.coarse_inverse() @ A, np.eye(A.shape[0]), atol=1e-11)


# ---------------------------------------------------------------- V-cycle
def vcycle_matrix(amg, N):
    return np.stack([amg.vcycle(e).ravel() for e in np.eye(N)], axis=1)


def test_vcycle_is_two_grid_operator():
    """M^-1 = (I - E) A^-1 with E = S^nu2 (I - P Ac^-1 P^T A) S^nu1,
    S = I - omega D^-1 A: the textbook two-grid error propagation."""
    sys = synth.density(4, 3, 2, seed=2)
    bsr, amg = hierarchy(sys, coarse_size=10, nu1=2, nu2=1)
    assert amg.levels == 2
    n = sys["n"]
    A = dense_from_bsr(amg.A(0))
    N = A.shape[0]
    Dinv = np.zeros_like(A)
    for i, blk in enumerate(amg.dinv(0)):
        Dinv[i * n:(i + 1) * n, i * n:(i + 1) * n] = blk
    S = np.eye(N) - 0.8 * Dinv @ A
    P = dense_from_bsr(amg.P(0))
    Ac = P.T @ A @ P
    CG = np.eye(N) - P @ np.linalg.solve(Ac, P.T @ A)
    E = S @ CG @ S @ S
    Minv_ref = (np.eye(N) - E) @ np.linalg.inv(A)
    M = vcycle_matrix(amg, N)
    assert np.allclose(M, Minv_ref, rtol=1e-10, atol=1e-11 * np.abs(Minv_ref).max())


def test_vcycle_linear_and_symmetric():
    sys = synth.density(4, seed=3)
    n = sys["n"]
    # symmetric matrix: lower = upper^T, symmetric diagonal blocks
    sys["lower"] = np.ascontiguousarray(np.transpose(sys["upper"], (0, 2, 1)))
    sys["diag"] = np.ascontiguousarray(0.5 * (sys["diag"] + np.transpose(sys["diag"], (0, 2, 1))))
    bsr, amg = hierarchy(sys, coarse_size=8, nu1=2, nu2=2)
    rng = np.random.default_rng(1)
    u = rng.standard_normal((bsr["rows"], n))
    v = rng.standard_normal((bsr["rows"], n))
    Mu, Mv = amg.vcycle(u), amg.vcycle(v)
    lin = amg.vcycle(2.0 * u - 3.0 * v)
    assert np.allclose(lin, 2.0 * Mu - 3.0 * Mv, rtol=1e-12, atol=1e-12 * np.abs(lin).max())
    assert np.dot(u.ravel(), Mv.ravel()) == pytest.approx(np.dot(v.ravel(), Mu.ravel()), rel=1e-11)


def test_one_level_cycle_is_exact_inverse():
    sys = synth.density(3, seed=1)
    bsr, amg = hierarchy(sys, coarse_size=10 ** 6)
    assert amg.levels == 1
    A = dense_from_bsr(amg.A(0))
    b = sys["b"]
    assert np.allclose(amg.vcycle(b).ravel(), np.linalg.solve(A, b.ravel()), rtol=1e-11, atol=1e-12)


def test_resetup_equals_fresh_setup_same_aggregates():
    sys = synth.density(6, seed=7)
    bsr, amg = hierarchy(sys)
    new = synth.perturb(sys, np.random.default_rng(1), 0.02)
    nb = oracle.ldu_to_bsr(new)
    assert amg.resetup(nb["val"]) == 0
    fresh = oracle.Amg(nb)
    # aggregation of the perturbed matrix may differ; compare where it does not
    same = all(np.array_equal(amg.P(l)["agg"], fresh.P(l)["agg"]) for l in range(min(amg.levels, fresh.levels) - 1))
    if same and amg.levels == fresh.levels:
        for l in range(amg.levels):
            assert np.array_equal(amg.A(l)["val"], fresh.A(l)["val"])
    # either way the resetup hierarchy is the Galerkin hierarchy of the new values
    for l in range(amg.levels - 1):
        Pd = dense_from_bsr(amg.P(l))
        ref = Pd.T @ dense_from_bsr(amg.A(l)) @ Pd
        assert np.allclose(dense_from_bsr(amg.A(l + 1)), ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    assert np.array_equal(amg.A(0)["val"], nb["val"])
