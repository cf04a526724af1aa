"""Oracle pins for the density-based assembly (Sec. 2.1, Eqs. approxJac1 /
approxJac2, pseudo-time term of Eq. discretBackward).

Pinned against: the Euler flux being homogeneous of degree one in Q
(J(Q, n) Q = F(Q, n)), central finite differences of F, the eigenvalues
V - c, V, V, V, V + c of J for a unit normal, linearity of J in n, the
closed form of lambda for equal states, the assembled blocks against a
finite-difference Jacobian of the frozen-lambda face residual
R_i = sum_f S/2 (F(Q_i, n) + F(Q_j, n) - lambda (Q_j - Q_i)) on a small mesh,
conservation (every block column sums to (sum_f lambda_f S_f / CFL) I) and
rejection of non-physical states.
"""
import numpy as np
import pytest

import oracle
from paper_2403_07882_b300 import synth

G = 1.4


def random_state(rng, mach=0.8):
    rho = rng.uniform(0.5, 2.0)
    u = rng.standard_normal(3) * mach
    p = rng.uniform(0.3, 2.0)
    return np.array([rho, *(rho * u), p / (G - 1) + 0.5 * rho * u @ u])


def unit(rng):
    n = rng.standard_normal(3)
    return n / np.linalg.norm(n)


def prims(Q):
    rho = Q[0]
    u = Q[1:4] / rho
    p = (G - 1) * (Q[4] - 0.5 * rho * u @ u)
    return rho, u, p


def test_flux_homogeneous_and_finite_differences():
    rng = np.random.default_rng(0)
    for _ in range(50):
        Q, n = random_state(rng), unit(rng) * rng.uniform(0.5, 2.0)
        F = oracle.euler_flux(Q, n, G)
        J = oracle.flux_jacobian(Q, n, G)
        assert np.allclose(J @ Q, F, rtol=1e-13, atol=1e-13 * np.abs(F).max())
        for k in range(5):
            h = 1e-6 * max(1.0, abs(Q[k]))
            e = np.zeros(5)
            e[k] = h
            fd = (oracle.euler_flux(Q + e, n, G) - oracle.euler_flux(Q - e, n, G)) / (2 * h)
            assert np.allclose(J[:, k], fd, rtol=1e-6, atol=1e-7 * np.abs(J).max()), k


def test_flux_definition_and_eigenvalues():
    rng = np.random.default_rng(1)
    for _ in range(30):
        Q, n = random_state(rng), unit(rng)
        rho, u, p = prims(Q)
        V = u @ n
        H = (Q[4] + p) / rho
        F = oracle.euler_flux(Q, n, G)
        assert np.allclose(F, [rho * V, *(rho * u * V + p * n), rho * H * V], rtol=1e-14)
        c = np.sqrt(G * p / rho)
        ev = np.sort(np.linalg.eigvals(oracle.flux_jacobian(Q, n, G)).real)
        assert np.allclose(ev, np.sort([V - c, V, V, V, V + c]), atol=1e-9 * (abs(V) + c))


def test_jacobian_linear_in_normal():
    rng = np.random.default_rng(2)
    Q = random_state(rng)
    n1, n2 = rng.standard_normal(3), rng.standard_normal(3)
    J1, J2 = oracle.flux_jacobian(Q, n1, G), oracle.flux_jacobian(Q, n2, G)
    assert np.array_equal(oracle.flux_jacobian(Q, -n1, G), -J1)
    assert np.allclose(oracle.flux_jacobian(Q, 2 * n1 - 3 * n2, G), 2 * J1 - 3 * J2, rtol=1e-13, atol=1e-13)
    # fluid at rest: continuity row (0, n, 0), energy row (0, H n, 0)
    Q0 = np.array([1.3, 0, 0, 0, 2.0])
    J0 = oracle.flux_jacobian(Q0, n1, G)
    H = (Q0[4] + (G - 1) * Q0[4]) / Q0[0]
    assert np.array_equal(J0[0], [0, *n1, 0])
    assert np.allclose(J0[4], [0, *(H * n1), 0], rtol=1e-15)


def test_lambda_closed_form_and_symmetry():
    rng = np.random.default_rng(3)
    for _ in range(20):
        Q, n = random_state(rng), unit(rng)
        rho, u, p = prims(Q)
        mu, pr, d = 1e-2, 0.72, 0.1
        lam = oracle.face_lambda(Q, Q, n, d, G, mu, pr)
        ref = abs(u @ n) + np.sqrt(G * p / rho) + max(4 / 3, G) * mu / (pr * rho * d)
        assert lam == pytest.approx(ref, rel=1e-13)
        Q2 = random_state(rng)
        assert oracle.face_lambda(Q, Q2, n, d, G, mu, pr) == oracle.face_lambda(Q2, Q, n, d, G, mu, pr)


def frozen_residual(fl, lam, Q):
    C = fl["n_cells"]
    R = np.zeros((C, 5))
    for f in range(fl["n_faces"]):
        i, j = fl["owner"][f], fl["neighbour"][f]
        n, S = fl["normal"][f], fl["area"][f]
        Fij = 0.5 * S * (oracle.euler_flux(Q[i], n, G) + oracle.euler_flux(Q[j], n, G) - lam[f] * (Q[j] - Q[i]))
        R[i] += Fij
        R[j] -= Fij
    return R


@pytest.mark.parametrize("skew", [False, True])
def test_assembly_is_jacobian_of_frozen_residual(skew):
    fl = synth.flow(3, 2, 2, seed=4, skew=skew)
    prm = dict(gamma=G, mu=1e-2, prandtl=0.72, cfl=5.0)
    st, diag, upper, lower = oracle.assemble_density(fl, **prm)
    assert st == 0
    C, F = fl["n_cells"], fl["n_faces"]
    lam = np.array([oracle.face_lambda(fl["Q"][fl["owner"][f]], fl["Q"][fl["neighbour"][f]], fl["normal"][f],
                                       fl["dist"][f], G, prm["mu"], prm["prandtl"]) for f in range(F)])
    tsum = np.zeros(C)
    np.add.at(tsum, fl["owner"], lam * fl["area"])
    np.add.at(tsum, fl["neighbour"], lam * fl["area"])
    A = np.zeros((5 * C, 5 * C))
    for c in range(C):
        A[5 * c:5 * c + 5, 5 * c:5 * c + 5] = diag[c] - tsum[c] / prm["cfl"] * np.eye(5)
    for f in range(F):
        i, j = fl["owner"][f], fl["neighbour"][f]
        A[5 * i:5 * i + 5, 5 * j:5 * j + 5] = upper[f]
        A[5 * j:5 * j + 5, 5 * i:5 * i + 5] = lower[f]
    Q = fl["Q"].copy()
    fd = np.zeros_like(A)
    for k in range(5 * C):
        h = 1e-6 * max(1.0, abs(Q.flat[k]))
        Qp, Qm = Q.copy(), Q.copy()
        Qp.flat[k] += h
        Qm.flat[k] -= h
        fd[:, k] = (frozen_residual(fl, lam, Qp) - frozen_residual(fl, lam, Qm)).ravel() / (2 * h)
    assert np.allclose(A, fd, rtol=1e-6, atol=1e-8 * np.abs(A).max())


@pytest.mark.parametrize("skew", [False, True])
def test_assembly_conservation(skew):
    fl = synth.flow(5, 4, 3, seed=6, skew=skew)
    cfl = 7.0
    st, diag, upper, lower = oracle.assemble_density(fl, cfl=cfl)
    assert st == 0
    C, o, nb = fl["n_cells"], fl["owner"], fl["neighbour"]
    colsum = diag.copy()
    np.add.at(colsum, nb, upper)   # upper[f] sits in column neighbour
    np.add.at(colsum, o, lower)    # lower[f] sits in column owner
    p = oracle.FLOW_DEFAULTS
    lam = np.array([oracle.face_lambda(fl["Q"][o[f]], fl["Q"][nb[f]], fl["normal"][f], fl["dist"][f], p["gamma"],
                                       p["mu"], p["prandtl"]) for f in range(fl["n_faces"])])
    tsum = np.zeros(C)
    np.add.at(tsum, o, lam * fl["area"])
    np.add.at(tsum, nb, lam * fl["area"])
    ref = (tsum / cfl)[:, None, None] * np.eye(5)
    scale = np.abs(diag).max()
    assert np.allclose(colsum, ref, rtol=0, atol=1e-13 * scale)


def test_assembly_rejects_invalid_states_and_parameters():
    fl = synth.flow(3, seed=1)
    bad = dict(fl, Q=fl["Q"].copy())
    bad["Q"][4, 0] = -1.0
    assert oracle.assemble_density(bad)[0] == 1
    bad = dict(fl, Q=fl["Q"].copy())
    bad["Q"][7, 4] = 0.1 * 0.5 * (bad["Q"][7, 1:4] ** 2).sum() / bad["Q"][7, 0]  # p < 0
    assert oracle.assemble_density(bad)[0] == 1
    assert oracle.assemble_density(fl, cfl=0.0)[0] == 1
    assert oracle.assemble_density(fl, gamma=1.0)[0] == 1
    assert oracle.assemble_density(fl)[0] == 0


def test_assembled_system_solves():
    """The assembled pseudo-time system is solved to 1e-8 by FGMRES and
    BiCGStab with the aggregation AMG (true residual recomputed here)."""
    fl = synth.flow(10, seed=2)
    st, diag, upper, lower = oracle.assemble_density(fl)
    assert st == 0
    sysm = dict(n_cells=fl["n_cells"], n_faces=fl["n_faces"], n=5, owner=fl["owner"], neighbour=fl["neighbour"],
                diag=diag, upper=upper, lower=lower, b=fl["b"])
    bsr = oracle.ldu_to_bsr(sysm)
    for solver in (0, 1):
        x, res, _ = oracle.solve(bsr, fl["b"], cfg=oracle.config(solver=solver))
        assert res["status"] == 0
        r = fl["b"] - oracle.spmv(bsr, x)
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(fl["b"])


def test_single_cell_and_single_face():
    """No faces: the diagonal block is zero (no face terms, no time term). One
    face: the two diagonal blocks and the two off-diagonal blocks are the
    four terms of Eqs. approxJac1/2 written out."""
    fl = synth.flow(1, 1, 1, seed=2)
    st, d, u, l = oracle.assemble_density(fl)
    assert st == 0 and u.shape == (0, 5, 5) and np.array_equal(d, np.zeros((1, 5, 5)))
    fl = synth.flow(2, 1, 1, seed=3)
    p = oracle.FLOW_DEFAULTS
    st, d, u, l = oracle.assemble_density(fl)
    assert st == 0
    n, S = fl["normal"][0], fl["area"][0]
    Qi, Qj = fl["Q"][0], fl["Q"][1]
    lam = oracle.face_lambda(Qi, Qj, n, fl["dist"][0], p["gamma"], p["mu"], p["prandtl"])
    Ji, Jj, I = oracle.flux_jacobian(Qi, n), oracle.flux_jacobian(Qj, n), np.eye(5)
    t = lam * S / p["cfl"]
    assert np.allclose(d[0], 0.5 * S * (Ji + lam * I) + t * I, rtol=1e-14, atol=1e-15)
    assert np.allclose(d[1], 0.5 * S * (-Jj + lam * I) + t * I, rtol=1e-14, atol=1e-15)
    assert np.allclose(u[0], 0.5 * S * (Jj - lam * I), rtol=1e-14, atol=1e-15)
    assert np.allclose(l[0], 0.5 * S * (-Ji - lam * I), rtol=1e-14, atol=1e-15)
