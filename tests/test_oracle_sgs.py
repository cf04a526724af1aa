"""Oracle pins for the multicolour block SGS (LU-SGS) preconditioner and
smoother (the CPU code's GMRES + LU-SGS, Sec. 2.1, and the GPU runs'
"GMRES with SGS preconditioner", Sec. 5): M = (D + L) D^-1 (D + U) with the
colour order of the DILU smoother.

Pinned against: a textbook symmetric block Gauss-Seidel (a forward sweep in
colour order then a backward sweep in reverse order, plain loops, from x = 0)
and a dense numpy solve with M; inside FGMRES every preconditioned vector
Z_j equals M^-1 V_j (Arnoldi hook); the AMG V-cycle with the SGS smoother
equals the two-grid error-propagation operator with S = I - M^-1 A; the
stored smoother factor equals D^-1; GMRES + SGS solves to 1e-8 (true
residual recomputed with numpy).
"""
import numpy as np
import pytest

import oracle
from paper_2403_07882_b300 import synth
from test_oracle_format import dense_from_bsr
from test_oracle_amg import hierarchy, vcycle_matrix

GENS = [lambda: synth.density(5, 4, 3, seed=1), lambda: synth.pressure(4, seed=2),
        lambda: synth.knn(5, seed=3), lambda: synth.random_graph(40, 120, 3, seed=4)]


def blocks(bsr):
    n, rp, ci, val = bsr["n"], bsr["row_ptr"], bsr["col"], bsr["val"]
    return {(i, ci[k]): val[k] for i in range(bsr["rows"]) for k in range(rp[i], rp[i + 1])}


def textbook_sgs(bsr, colour, r):
    """Symmetric block Gauss-Seidel from x = 0: forward over the rows sorted
    by (colour, index), each row solved with the latest values, then backward
    over the reverse order."""
    n, rows = bsr["n"], bsr["rows"]
    B = blocks(bsr)
    nbrs = [[j for (i2, j) in B if i2 == i] for i in range(rows)]
    order = sorted(range(rows), key=lambda i: (colour[i], i))
    x = np.zeros((rows, n))

    def relax(i):
        s = r[i].copy()
        for j in nbrs[i]:
            if j != i:
                s -= B[(i, j)] @ x[j]
        x[i] = np.linalg.solve(B[(i, i)], s)

    for i in order:
        relax(i)
    for i in reversed(order):
        relax(i)
    return x


def dense_sgs(bsr, colour):
    n = bsr["n"]
    A = dense_from_bsr(bsr)
    D = np.zeros_like(A)
    L = np.zeros_like(A)
    U = np.zeros_like(A)
    for (i, j), blk in blocks(bsr).items():
        s, t = slice(i * n, (i + 1) * n), slice(j * n, (j + 1) * n)
        if i == j:
            D[s, t] = blk
        elif colour[j] < colour[i]:
            L[s, t] = blk
        elif colour[j] > colour[i]:
            U[s, t] = blk
    return A, (D + L) @ np.linalg.inv(D) @ (D + U)


@pytest.mark.parametrize("gen", GENS)
def test_sgs_apply_is_symmetric_gauss_seidel(gen):
    bsr = oracle.ldu_to_bsr(gen())
    nc, col = oracle.colour(bsr)
    dinv = np.stack([np.linalg.inv(b) for b in
                     (dense_from_bsr(bsr).reshape(bsr["rows"], bsr["n"], bsr["rows"], bsr["n"])
                      [i, :, i, :] for i in range(bsr["rows"]))])
    r = np.random.default_rng(5).standard_normal((bsr["rows"], bsr["n"]))
    z = oracle.dilu_apply(bsr, col, dinv, r)
    assert np.allclose(z, textbook_sgs(bsr, col, r), rtol=1e-11, atol=1e-11 * np.abs(z).max())
    A, M = dense_sgs(bsr, col)
    assert np.allclose(z.ravel(), np.linalg.solve(M, r.ravel()), rtol=1e-10, atol=1e-10 * np.abs(z).max())


def test_fgmres_uses_sgs_preconditioner():
    sys = synth.density(4, 3, 3, seed=6)
    bsr = oracle.ldu_to_bsr(sys)
    cfg = oracle.config(precond=3)
    done, V, Z, H = oracle.arnoldi(bsr, sys["b"], 6, cfg=cfg)
    nc, col = oracle.colour(bsr)
    A, M = dense_sgs(bsr, col)
    for j in range(done):
        assert np.allclose(Z[j], np.linalg.solve(M, V[j]), rtol=1e-10, atol=1e-12)
    # Arnoldi relation A Z_j = V_{j+1} H_j
    assert np.allclose(A @ Z[:done].T, V[:done + 1].T @ H[:done + 1, :done], atol=1e-10)


def test_sgs_smoother_two_grid_operator():
    sys = synth.density(4, 3, 2, seed=2)
    bsr, amg = hierarchy(sys, coarse_size=10, nu1=2, nu2=1, smoother=2)
    assert amg.levels == 2
    nc, col, einv = amg.dilu(0)
    assert nc > 0
    assert np.array_equal(einv, amg.dinv(0))
    A, M = dense_sgs(amg.A(0), col)
    N = A.shape[0]
    S = np.eye(N) - np.linalg.solve(M, A)
    P = dense_from_bsr(amg.P(0))
    CG = np.eye(N) - P @ np.linalg.solve(P.T @ A @ P, P.T @ A)
    Minv_ref = (np.eye(N) - S @ CG @ S @ S) @ np.linalg.inv(A)
    assert np.allclose(vcycle_matrix(amg, N), Minv_ref, rtol=1e-9, atol=1e-10 * np.abs(Minv_ref).max())


@pytest.mark.parametrize("gen", [lambda: synth.density(10, seed=1), lambda: synth.pressure(8, seed=2)])
def test_gmres_sgs_and_amg_sgs_solve(gen):
    sys = gen()
    bsr = oracle.ldu_to_bsr(sys)
    A = dense_from_bsr(bsr)
    its = {}
    for name, cfg in (("gmres+sgs", oracle.config(precond=3, maxiter=2000)),
                      ("gmres+amg(sgs)", oracle.config(smoother=2)),
                      ("gmres+jacobi", oracle.config(precond=2, maxiter=2000))):
        x, res, _ = oracle.solve(bsr, sys["b"], cfg=cfg)
        assert res["status"] == 0, name
        r = sys["b"].ravel() - A @ x.ravel()
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(sys["b"]), name
        its[name] = res["iters"]
    assert its["gmres+sgs"] < its["gmres+jacobi"]
    assert its["gmres+amg(sgs)"] < its["gmres+sgs"]


def test_sgs_beyond_128_colours_is_block_jacobi():
    """A complete graph of 130 cells needs 130 colours, more than the 128
    allowed: the SGS preconditioner falls back to one block-Jacobi solve."""
    m, n = 130, 2
    rng = np.random.default_rng(9)
    rows = [(i, j) for i in range(m) for j in range(i + 1, m)]
    owner = np.array([i for i, _ in rows], np.int32)
    nb = np.array([j for _, j in rows], np.int32)
    F = owner.size
    diag = np.repeat((4.0 * m * np.eye(n))[None], m, 0) + rng.standard_normal((m, n, n))
    sys_ = dict(n_cells=m, n_faces=F, n=n, owner=owner, neighbour=nb, diag=diag,
                upper=0.1 * rng.standard_normal((F, n, n)), lower=0.1 * rng.standard_normal((F, n, n)),
                b=rng.standard_normal((m, n)))
    bsr = oracle.ldu_to_bsr(sys_)
    nc, _ = oracle.colour(bsr)
    assert nc == -1
    done, V, Z, H = oracle.arnoldi(bsr, sys_["b"], 3, cfg=oracle.config(precond=3))
    Dinv = np.linalg.inv(diag)
    for j in range(done):
        assert np.allclose(Z[j].reshape(m, n), np.einsum("iab,ib->ia", Dinv, V[j].reshape(m, n)), rtol=1e-12,
                           atol=1e-14)
