"""GPU parity of the multicolour block SGS (LU-SGS form (D + L) D^-1 (D + U))
preconditioner and AMG smoother: colourings and factors (E = D) bit-exact with
the CPU reference; one preconditioner application and the V-cycle with the
SGS smoother at 1e-12 in FP64 and within FP32 / BF16 storage tolerance;
GMRES + SGS and BiCGStab + SGS solves to 1e-8 recomputed on the CPU, FP64
iteration counts within 2 of the reference's."""
import numpy as np
import pytest

import oracle
from paper_2403_07882_b300 import bcs, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
SGS = bcs.BCS_SMOOTH_SGS

CASES = [
    ("density 12^3", lambda: synth.density(12, seed=0), {}),
    ("pressure 10^3", lambda: synth.pressure(10, seed=1), {}),
    ("knn 10^3", lambda: synth.knn(10, seed=2), {}),
    ("random n=3", lambda: synth.random_graph(400, 1500, 3, seed=5), dict(coarse_size=8)),
    ("density 24^3", lambda: synth.density(24, seed=4), {}),
]
TOLS = ((bcs.BCS_PREC_FP64, None), (bcs.BCS_PREC_FP32, 2e-5), (bcs.BCS_PREC_BF16, 5e-2))


def close(z, z_ref, tol):
    if tol is None:
        return np.abs(z - z_ref).max() <= 1e-12 * np.abs(z_ref).max()
    return np.linalg.norm(z - z_ref) <= tol * np.linalg.norm(z_ref)


@pytest.mark.parametrize("name,gen,kw", CASES, ids=[c[0] for c in CASES])
def test_sgs_smoother_factor_and_vcycle(name, gen, kw):
    system = gen()
    amg = oracle.Amg(oracle.ldu_to_bsr(system), oracle.config(smoother=2, **kw))
    assert amg.status == 0
    v = np.random.default_rng(6).standard_normal(system["b"].shape)
    z_ref = amg.vcycle(v)
    for prec, tol in TOLS:
        with bcs.Solver(system["n"], precision=prec, smoother=SGS, **kw) as s:
            s.load(system, device=DEV)
            if prec == bcs.BCS_PREC_FP64:
                for l in range(amg.levels):
                    nc, col, einv = s.dilu(l)
                    nr, col_r, einv_r = amg.dilu(l)
                    assert nc == nr
                    if nc > 0:
                        assert np.array_equal(col, col_r) and np.array_equal(einv, einv_r)
                        assert np.array_equal(einv, amg.dinv(l))
            z = s.precond(torch.from_numpy(v).to(DEV)).cpu().numpy()
        assert close(z, z_ref, tol), (name, prec)


@pytest.mark.parametrize("name,gen,kw", CASES, ids=[c[0] for c in CASES])
def test_sgs_preconditioner_apply(name, gen, kw):
    system = gen()
    bsr = oracle.ldu_to_bsr(system)
    nc, col = oracle.colour(bsr)
    dinv = oracle.Amg(bsr, oracle.config(precond=1)).dinv(0)
    v = np.random.default_rng(7).standard_normal(system["b"].shape)
    z_ref = oracle.dilu_apply(bsr, col, dinv, v)
    for prec, tol in TOLS:
        with bcs.Solver(system["n"], precision=prec, precond=bcs.BCS_PC_SGS) as s:
            s.load(system, device=DEV)
            assert s.levels == 1
            z = s.precond(torch.from_numpy(v).to(DEV)).cpu().numpy()
        assert close(z, z_ref, tol), (name, prec)


@pytest.mark.parametrize("solver", [bcs.BCS_FGMRES, bcs.BCS_BICGSTAB], ids=["fgmres", "bicgstab"])
@pytest.mark.parametrize("gen", [lambda: synth.density(16, seed=0), lambda: synth.pressure(12, seed=1),
                                 lambda: synth.knn(12, seed=3)], ids=["density16", "pressure12", "knn12"])
def test_sgs_solves(gen, solver):
    system = gen()
    ref = oracle.ldu_to_bsr(system)
    _, res_r, _ = oracle.solve(ref, system["b"], cfg=oracle.config(precond=3, solver=solver, maxiter=3000))
    assert res_r["status"] == 0
    for prec in (bcs.BCS_PREC_FP64, bcs.BCS_PREC_FP32):
        with bcs.Solver(system["n"], solver=solver, precond=bcs.BCS_PC_SGS, precision=prec, maxiter=3000) as s:
            s.load(system, device=DEV)
            x, st, res = s.solve(torch.from_numpy(system["b"]).to(DEV))
            assert st == bcs.BCS_OK, res
            xh = x.cpu().numpy()
        r = system["b"] - oracle.spmv(ref, xh)
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(system["b"])
        if prec == bcs.BCS_PREC_FP64:
            assert abs(res["iters"] - res_r["iters"]) <= 2, (res["iters"], res_r["iters"])
    # AMG with the SGS smoother
    with bcs.Solver(system["n"], solver=solver, smoother=SGS) as s:
        s.load(system, device=DEV)
        x, st, res = s.solve(torch.from_numpy(system["b"]).to(DEV))
        assert st == bcs.BCS_OK, res
    r = system["b"] - oracle.spmv(ref, x.cpu().numpy())
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(system["b"])


def test_sgs_beyond_128_colours_is_block_jacobi():
    """130 mutually coupled cells need more than the 128 colours allowed: the
    SGS preconditioner is then one block-Jacobi solve, as in the reference."""
    m, n = 130, 2
    rng = np.random.default_rng(9)
    pairs = [(i, j) for i in range(m) for j in range(i + 1, m)]
    owner = np.array([i for i, _ in pairs], np.int32)
    nb = np.array([j for _, j in pairs], np.int32)
    F = owner.size
    diag = np.repeat((4.0 * m * np.eye(n))[None], m, 0) + rng.standard_normal((m, n, n))
    system = dict(n_cells=m, n_faces=F, n=n, owner=owner, neighbour=nb, diag=diag,
                  upper=0.1 * rng.standard_normal((F, n, n)), lower=0.1 * rng.standard_normal((F, n, n)),
                  b=rng.standard_normal((m, n)))
    v = rng.standard_normal((m, n))
    z_ref = np.einsum("iab,ib->ia", np.linalg.inv(diag), v)
    with bcs.Solver(n, precond=bcs.BCS_PC_SGS, precision=bcs.BCS_PREC_FP64) as s:
        s.load(system, device=DEV)
        assert s.dilu(0)[0] <= 0
        z = s.precond(torch.from_numpy(v).to(DEV)).cpu().numpy()
    assert np.allclose(z, z_ref, rtol=1e-12, atol=1e-14)
