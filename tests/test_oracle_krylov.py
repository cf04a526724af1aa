"""Oracle pins for the Krylov solvers (GMRES of Saad & Schultz, Sec. 2; the
GPU solvers of Sec. 2.3: GMRES and BiCGStab with AMG).

Pinned against: the Arnoldi relation and orthonormality, brute-force
least-squares minimality over the Krylov space (numpy lstsq), termination in
N steps, one-iteration convergence with an exact preconditioner, and the true
residual recomputed with numpy.
"""
import numpy as np
import pytest

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
