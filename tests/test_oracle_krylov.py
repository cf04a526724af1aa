"""Oracle pins for the Krylov solvers (GMRES of Saad & Schultz, Sec. 2; the
GPU solvers of Sec. 2.3: GMRES and BiCGStab with AMG).

Pinned against: the Arnoldi relation and orthonormality, brute-force
least-squares minimality over the Krylov space (numpy lstsq) for one cycle
and for a chain of restarted cycles, termination in N steps, one-iteration
convergence with an exact preconditioner, the true residual recomputed with
numpy, BiCGStab's recurrence residual against the true residual of every
iterate, and BiCGStab's iterates against SciPy's independent implementation
of the same method (van der Vorst's BiCGStab, right preconditioned, shadow
residual r_0).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

import oracle
from paper_2403_07882_b300 import synth
from test_oracle_format import dense_from_bsr


def test_arnoldi_relation():
    sys = synth.density(6, seed=2)
    bsr = oracle.ldu_to_bsr(sys)
    cfg = oracle.config(coarse_size=8)
    amg = oracle.Amg(bsr, cfg)
    assert amg.levels >= 3
    j = 8
    done, V, Z, H = oracle.arnoldi(bsr, sys["b"], j, cfg, amg)
    assert done == j
    A = dense_from_bsr(bsr)
    lhs = A @ Z.T
    rhs = V.T @ H
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(lhs).max()
    assert np.allclose(V @ V.T, np.eye(j + 1), atol=1e-13)
    # flexible GMRES: Z_j is the preconditioner applied to V_j
    for k in range(j):
        assert np.allclose(Z[k], amg.vcycle(V[k]).ravel(), rtol=1e-14, atol=1e-15)


def test_gmres_residual_is_krylov_minimum():
    """M = I, x0 = 0: after j steps the residual is min ||b - A y|| over
    y in K_j(A, b); brute force with an orthonormal Krylov basis (numpy QR)."""
    sys = synth.random_graph(8, 12, 2, seed=3)
    bsr = oracle.ldu_to_bsr(sys)
    N = bsr["rows"] * bsr["n"]
    A = dense_from_bsr(bsr)
    b = sys["b"].ravel()
    cfg = oracle.config(precond=1, restart=N, maxiter=N, tol=1e-300)
    x, res, hist = oracle.solve(bsr, b, cfg=cfg, hist_len=N)
    # orthonormal basis of K_j grown by numpy QR: span{Q_j, A q_j} = K_{j+1}
    Q = (b / np.linalg.norm(b))[:, None]
    for j in range(1, N):
        y, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
        rmin = np.linalg.norm(b - A @ Q @ y) / np.linalg.norm(b)
        assert hist[j - 1] == pytest.approx(rmin, rel=1e-6, abs=1e-12)
        Q, _ = np.linalg.qr(np.column_stack([Q, A @ Q[:, -1]]))
    # N steps reach the exact solution
    assert np.allclose(x.ravel(), np.linalg.solve(A, b), rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("solver", [0, 1])
def test_exact_preconditioner_one_iteration(solver):
    sys = synth.density(3, seed=4)
    bsr = oracle.ldu_to_bsr(sys)
    cfg = oracle.config(solver=solver, coarse_size=10 ** 6)
    x, res, _ = oracle.solve(bsr, sys["b"], cfg=cfg)
    assert res["status"] == 0 and res["iters"] == 1
    assert res["rel_res_final"] < 1e-12


def true_rel_residual(bsr, b, x):
    A = dense_from_bsr(bsr) if bsr["rows"] * bsr["n"] <= 4000 else None
    if A is not None:
        r = b.ravel() - A @ x.ravel()
    else:
        import scipy.sparse as sp
        n = bsr["n"]
        rows = np.repeat(np.arange(bsr["rows"]), np.diff(bsr["row_ptr"]))
        ii = (rows[:, None, None] * n + np.arange(n)[None, :, None]).repeat(n, 2)
        jj = (bsr["col"][:, None, None] * n + np.arange(n)[None, None, :]).repeat(n, 1)
        M = sp.csr_matrix((bsr["val"].ravel(), (ii.ravel(), jj.ravel())))
        r = b.ravel() - M @ x.ravel()
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("gen", [lambda: synth.density(16, seed=0), lambda: synth.pressure(16, seed=1)])
def test_end_to_end_true_residual(solver, gen):
    sys = gen()
    bsr = oracle.ldu_to_bsr(sys)
    cfg = oracle.config(solver=solver)
    x, res, _ = oracle.solve(bsr, sys["b"], cfg=cfg)
    assert res["status"] == 0
    rel = true_rel_residual(bsr, sys["b"], x)
    assert rel <= 1e-8
    assert rel == pytest.approx(res["rel_res_final"], rel=1e-6)


def test_zero_rhs_and_maxiter():
    sys = synth.density(4, seed=5)
    bsr = oracle.ldu_to_bsr(sys)
    x, res, _ = oracle.solve(bsr, np.zeros_like(sys["b"]), x0=np.ones(sys["b"].size))
    assert res["status"] == 0 and np.all(x == 0)
    x, res, _ = oracle.solve(bsr, sys["b"], cfg=oracle.config(maxiter=1, precond=1))
    assert res["status"] == 4 and res["iters"] == 1


def test_singular_block_reported():
    sys = synth.density(3, seed=6)
    sys["diag"][4] = 0.0
    bsr = oracle.ldu_to_bsr(sys)
    x, res, _ = oracle.solve(bsr, sys["b"])
    assert res["status"] == 6


def test_block_jacobi_and_none_preconditioners_converge():
    sys = synth.density(6, seed=8)
    bsr = oracle.ldu_to_bsr(sys)
    for pc in (1, 2):
        x, res, _ = oracle.solve(bsr, sys["b"], cfg=oracle.config(precond=pc))
        assert res["status"] == 0 and true_rel_residual(bsr, sys["b"], x) <= 1e-8


def test_restarted_gmres_cycles_are_krylov_minima():
    """FGMRES(3), M = I, x0 = 0: within each restart cycle c the residual
    after j steps is min ||r_c - A y|| over y in K_j(A, r_c), r_c the true
    residual the cycle starts from. Brute force: numpy builds each cycle's
    Krylov basis by QR, solves the least-squares problem and carries its own
    iterate to the next cycle."""
    for sys in (synth.random_graph(8, 12, 2, seed=3), synth.random_graph(12, 20, 3, seed=5)):
        bsr = oracle.ldu_to_bsr(sys)
        A = dense_from_bsr(bsr)
        b = sys["b"].ravel()
        N, m, cycles = A.shape[0], 3, 5
        assert N >= 12
        cfg = oracle.config(precond=1, restart=m, maxiter=m * cycles, tol=1e-300)
        x, res, hist = oracle.solve(bsr, b, cfg=cfg, hist_len=m * cycles)
        assert res["iters"] == m * cycles and res["restarts"] == cycles - 1
        xc = np.zeros(N)
        bn = np.linalg.norm(b)
        ref = []
        for _ in range(cycles):
            r = b - A @ xc
            Q = (r / np.linalg.norm(r))[:, None]
            for j in range(1, m + 1):
                y, *_ = np.linalg.lstsq(A @ Q, r, rcond=None)
                ref.append(np.linalg.norm(r - A @ Q @ y) / bn)
                if j < m:
                    Q, _ = np.linalg.qr(np.column_stack([Q, A @ Q[:, -1]]))
            xc = xc + Q @ y
        np.testing.assert_allclose(hist, ref, rtol=1e-9, atol=0)
        # a restarted method loses the minimality over the whole space: the
        # chain ends above the unrestarted minimum of the same step count
        assert np.linalg.norm(x.ravel() - xc) <= 1e-12 * np.linalg.norm(xc)


def _bicgstab_cases():
    return [synth.density(3, seed=4), synth.random_graph(30, 60, 4, seed=3), synth.random_graph(36, 80, 5, seed=7)]


@pytest.mark.parametrize("case", range(3))
def test_bicgstab_recurrence_equals_true_residual(case):
    """The residual BiCGStab carries by recurrence (r_k = s - omega t) is the
    true residual b - A x_k of its iterate, at every iteration, up to
    rounding (Sec. 2.3's PBiCGStab; van der Vorst's update of x and r)."""
    sys = _bicgstab_cases()[case]
    bsr = oracle.ldu_to_bsr(sys)
    A = dense_from_bsr(bsr)
    b = sys["b"].ravel()
    for precond in (1, 2, 0):
        cfg = oracle.config(solver=1, precond=precond, tol=1e-12, maxiter=80, coarse_size=8)
        amg = oracle.Amg(bsr, cfg) if precond == 0 else None
        x, res, xs, rs = oracle.bicgstab_trace(bsr, b, cfg, amg=amg)
        assert res["status"] == 0 and res["restarts"] == 0 and len(xs) == res["iters"] >= 2
        for k in range(len(xs)):
            drift = np.linalg.norm(rs[k] - (b - A @ xs[k]))
            assert drift <= 1e-10 * np.linalg.norm(b), (precond, k, drift)
        assert np.array_equal(xs[-1], x.ravel())


def _block_jacobi_operator(bsr):
    n, rows = bsr["n"], bsr["rows"]
    D = np.zeros((rows, n, n))
    for i in range(rows):
        k = bsr["row_ptr"][i] + int(np.nonzero(bsr["col"][bsr["row_ptr"][i]:bsr["row_ptr"][i + 1]] == i)[0][0])
        D[i] = np.linalg.inv(bsr["val"][k])
    return sla.LinearOperator((rows * n, rows * n), matvec=lambda v: np.einsum("irc,ic->ir", D, v.reshape(rows, n)).ravel())


@pytest.mark.parametrize("case", range(3))
@pytest.mark.parametrize("precond", [1, 2])
def test_bicgstab_iterates_match_scipy(case, precond):
    """Same method, independent code: SciPy's bicgstab (shadow residual r_0,
    beta = (rho / rho_old)(alpha / omega), omega = (t, s) / (t, t), right
    preconditioned: x += alpha M p + omega M s). Without a preconditioner and
    with one block-Jacobi solve z = D^-1 v as M, every iterate x_k agrees to
    rounding, and so do the residual norms while they are above the rounding
    floor."""
    sys = _bicgstab_cases()[case]
    bsr = oracle.ldu_to_bsr(sys)
    A = dense_from_bsr(bsr)
    b = sys["b"].ravel()
    assert A.shape[0] <= 200
    cfg = oracle.config(solver=1, precond=precond, tol=1e-13, maxiter=60)
    x, res, xs, rs = oracle.bicgstab_trace(bsr, b, cfg)
    sx = []
    M = _block_jacobi_operator(bsr) if precond == 2 else None
    sla.bicgstab(A, b, x0=np.zeros_like(b), rtol=1e-13, atol=0.0, maxiter=60, M=M,
                 callback=lambda xk: sx.append(xk.copy()))
    # SciPy calls back after full steps only; the oracle also records the
    # half step that ends the solve
    assert len(sx) >= 5 and len(xs) - 1 <= len(sx) <= len(xs)
    bn = np.linalg.norm(b)
    for k in range(len(sx)):
        assert np.linalg.norm(xs[k] - sx[k]) <= 1e-10 * np.linalg.norm(sx[k]), k
        ro, rsc = np.linalg.norm(b - A @ xs[k]) / bn, np.linalg.norm(b - A @ sx[k]) / bn
        if rsc > 1e-7:
            assert ro == pytest.approx(rsc, rel=1e-8), k


def test_openmp_build_gives_identical_results():
    """The OpenMP build of the oracle (used as the all-cores CPU baseline)
    splits only loops with disjoint outputs, so its solves equal the
    single-threaded build's bit for bit."""
    sys = synth.density(10, seed=3)
    bsr = oracle.ldu_to_bsr(sys)
    outs = []
    try:
        for omp in (False, True):
            oracle.use_openmp(omp)
            row = []
            for solver in (0, 1):
                cfg = oracle.config(solver=solver)
                x, res, _ = oracle.solve(bsr, sys["b"], cfg=cfg)
                assert res["status"] == 0
                row.append((x, res["iters"]))
            outs.append(row)
    finally:
        oracle.use_openmp(False)
    for (xa, ia), (xb, ib) in zip(*outs):
        assert ia == ib and np.array_equal(xa, xb)
