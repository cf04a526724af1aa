"""GPU parity of the Krylov solves (Sec. 2.3: GMRES / BiCGStab with AMG):
every GPU solution reaches the true relative residual 1e-8, recomputed on
the CPU with the FP64 reference SpMV; the reference solver reaches the same
tolerance on the same system; the solution difference is reported per case.
"""
import numpy as np
import pytest

import oracle
from paper_2403_07882_b300 import bcs, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def true_rel(ref, b, x):
    r = b - oracle.spmv(ref, x)
    return np.linalg.norm(r) / np.linalg.norm(b)


def gpu_solve(system, x0=None, device=True, **cfg):
    with bcs.Solver(system["n"], **cfg) as s:
        s.load(system, device=DEV if device else None)
        if device:
            b = torch.from_numpy(system["b"]).to(DEV)
            x = torch.zeros_like(b) if x0 is None else torch.from_numpy(x0).to(DEV)
            x, st, res = s.solve(b, x)
            x = x.cpu().numpy()
        else:
            x = np.zeros_like(system["b"]) if x0 is None else x0.copy()
            x, st, res = s.solve(system["b"], x)
    return x, st, res


SOLVES = [
    ("c1 density 16^3 fgmres fp32", lambda: synth.density(16, seed=0), dict()),
    ("c1 density 16^3 fgmres fp64", lambda: synth.density(16, seed=0), dict(precision=bcs.BCS_PREC_FP64)),
    ("c1 density 16^3 fgmres bf16", lambda: synth.density(16, seed=0), dict(precision=bcs.BCS_PREC_BF16)),
    ("c1 density 16^3 bicgstab fp32", lambda: synth.density(16, seed=0), dict(solver=bcs.BCS_BICGSTAB)),
    ("pressure 16^3 bicgstab fp32", lambda: synth.pressure(16, seed=1), dict(solver=bcs.BCS_BICGSTAB)),
    ("pressure 16^3 fgmres fp32", lambda: synth.pressure(16, seed=1), dict()),
    ("pressure 16^3 bicgstab fp64", lambda: synth.pressure(16, seed=1),
     dict(solver=bcs.BCS_BICGSTAB, precision=bcs.BCS_PREC_FP64)),
    ("density 12^3 smoothed P", lambda: synth.density(12, seed=3), dict(pmode=bcs.BCS_P_SMOOTHED)),
    ("random n=3", lambda: synth.random_graph(500, 1500, 3, seed=2), dict(coarse_size=16)),
]


@pytest.mark.parametrize("name,gen,cfg", SOLVES, ids=[c[0] for c in SOLVES])
def test_solve_reaches_tolerance(name, gen, cfg):
    system = gen()
    ref = oracle.ldu_to_bsr(system)
    x, st, res = gpu_solve(system, **cfg)
    assert st == bcs.BCS_OK, res
    rel = true_rel(ref, system["b"], x)
    assert rel <= 1e-8, rel
    assert rel == pytest.approx(res["rel_res_final"], rel=1e-5, abs=1e-14)
    ocfg = oracle.config(**{k: v for k, v in cfg.items() if k != "precision"})
    xo, ores, _ = oracle.solve(ref, system["b"], cfg=ocfg)
    assert ores["status"] == 0 and true_rel(ref, system["b"], xo) <= 1e-8
    if cfg.get("precision") == bcs.BCS_PREC_FP64:
        # FP64 everywhere: the same iteration count as the reference (+-1)
        assert abs(res["iters"] - ores["iters"]) <= 1, (res["iters"], ores["iters"])
    dx = np.linalg.norm(x - xo) / np.linalg.norm(xo)
    print(f"{name}: iters gpu={res['iters']} ref={ores['iters']} rel={rel:.2e} |dx|/|x|={dx:.2e}")


def test_host_memory_path_matches_device():
    system = synth.density(12, seed=1)
    xd, st1, r1 = gpu_solve(system, device=True)
    xh, st2, r2 = gpu_solve(system, device=False)
    assert st1 == st2 == bcs.BCS_OK
    assert np.array_equal(xd, xh) and r1["iters"] == r2["iters"]


def test_warm_start_and_zero_rhs():
    system = synth.density(10, seed=2)
    ref = oracle.ldu_to_bsr(system)
    x, st, res = gpu_solve(system)
    x2, st2, res2 = gpu_solve(system, x0=x)
    assert st2 == bcs.BCS_OK and res2["iters"] <= 1
    z = dict(system)
    z["b"] = np.zeros_like(system["b"])
    x3, st3, res3 = gpu_solve(z, x0=np.ones_like(system["b"]))
    assert st3 == bcs.BCS_OK and np.all(x3 == 0)


def test_maxiter_and_preconditioner_variants():
    system = synth.density(8, seed=4)
    ref = oracle.ldu_to_bsr(system)
    x, st, res = gpu_solve(system, maxiter=1, precond=bcs.BCS_PC_NONE)
    assert st == bcs.BCS_NOT_CONVERGED and res["iters"] == 1
    for pc in (bcs.BCS_PC_NONE, bcs.BCS_PC_JACOBI):
        for solver in (bcs.BCS_FGMRES, bcs.BCS_BICGSTAB):
            x, st, res = gpu_solve(system, precond=pc, solver=solver)
            assert st == bcs.BCS_OK and true_rel(ref, system["b"], x) <= 1e-8


def test_exact_preconditioner_one_iteration():
    system = synth.density(3, seed=4)
    for solver in (bcs.BCS_FGMRES, bcs.BCS_BICGSTAB):
        x, st, res = gpu_solve(system, solver=solver, coarse_size=10 ** 6, precision=bcs.BCS_PREC_FP64)
        assert st == bcs.BCS_OK and res["iters"] == 1


def test_state_errors():
    with bcs.Solver(5) as s:
        with pytest.raises(bcs.BcsError) as e:
            s.solve(np.ones((4, 5)))
        assert e.value.status == bcs.BCS_ESTATE
        with pytest.raises(bcs.BcsError) as e:
            s.set_values(np.ones((4, 5, 5)), np.ones((3, 5, 5)), np.ones((3, 5, 5)))
        assert e.value.status == bcs.BCS_ESTATE


def test_values_only_resetup_sequence():
    """Alg. 1: first iteration full setup, later iterations replace values on
    the fixed sparsity. Ten 2% perturbations, each solved to 1e-8."""
    system = synth.density(16, seed=3)
    rng = np.random.default_rng(31)
    with bcs.Solver(5) as s:
        s.load(system, device=DEV)
        agg0 = s.level(0)["agg"].copy()
        b = torch.from_numpy(system["b"]).to(DEV)
        for it in range(10):
            system = synth.perturb(system, rng, 0.02)
            s.set_values(*(torch.from_numpy(system[k]).to(DEV) for k in ("diag", "upper", "lower")))
            assert np.array_equal(s.level(0)["agg"], agg0)
            x, st, res = s.solve(b)
            assert st == bcs.BCS_OK
            assert true_rel(oracle.ldu_to_bsr(system), system["b"], x.cpu().numpy()) <= 1e-8


def test_full_size_128cube_mixed_solve():
    """The benchmark workload: 128^3 density-based 5x5 system, FGMRES(30)
    with FP32 AMG to 1e-8; true residual recomputed on the CPU."""
    system = synth.density(128, seed=2)
    ref = oracle.ldu_to_bsr(system)
    x, st, res = gpu_solve(system)
    assert st == bcs.BCS_OK, res
    assert true_rel(ref, system["b"], x) <= 1e-8


RESTARTS = [
    ("density 16^3 m=5", lambda: synth.density(16, seed=0), dict(restart=5)),
    ("pressure 12^3 m=5", lambda: synth.pressure(12, seed=1), dict(restart=5)),
    ("pressure 12^3 m=3", lambda: synth.pressure(12, seed=1), dict(restart=3)),
    ("density 12^3 m=2 no AMG", lambda: synth.density(12, seed=4), dict(restart=2, precond=bcs.BCS_PC_JACOBI)),
]


@pytest.mark.parametrize("name,gen,cfg", RESTARTS, ids=[c[0] for c in RESTARTS])
def test_restarted_fgmres_fp64_matches_oracle(name, gen, cfg):
    """FGMRES(m) with m below the iteration count (GMRES restarted after m
    steps from the true residual, Sec. 2), all in FP64: the GPU restarts as
    often as the oracle, takes the same number of iterations (+-1) and
    reaches the true relative residual 1e-8 recomputed on the CPU."""
    system = gen()
    ref = oracle.ldu_to_bsr(system)
    xo, ores, _ = oracle.solve(ref, system["b"], cfg=oracle.config(**cfg))
    assert ores["status"] == 0 and ores["restarts"] >= 1
    x, st, res = gpu_solve(system, precision=bcs.BCS_PREC_FP64, **cfg)
    assert st == bcs.BCS_OK, res
    assert abs(res["iters"] - ores["iters"]) <= 1, (res["iters"], ores["iters"])
    assert abs(res["restarts"] - ores["restarts"]) <= 1, (res["restarts"], ores["restarts"])
    assert res["restarts"] >= 1
    rel = true_rel(ref, system["b"], x)
    assert rel <= 1e-8
    dx = np.linalg.norm(x - xo) / np.linalg.norm(xo)
    print(f"{name}: iters gpu={res['iters']} ref={ores['iters']} restarts gpu={res['restarts']} "
          f"ref={ores['restarts']} |dx|/|x|={dx:.2e}")


@pytest.mark.parametrize("solver", [bcs.BCS_FGMRES, bcs.BCS_BICGSTAB])
@pytest.mark.parametrize("precision", [bcs.BCS_PREC_FP64, bcs.BCS_PREC_FP32])
def test_coarse_smoother_sweeps_solve(solver, precision):
    """Coarsest level without the dense inverse (coarse_dense_max = 1: eight
    block-Jacobi sweeps there instead): solves still reach 1e-8, FP64 in the
    oracle's iteration count (+-1)."""
    system = synth.pressure(12, seed=1)
    cfg = dict(coarse_dense_max=1, solver=solver)
    ref = oracle.ldu_to_bsr(system)
    xo, ores, _ = oracle.solve(ref, system["b"], cfg=oracle.config(**cfg))
    assert ores["status"] == 0
    x, st, res = gpu_solve(system, precision=precision, **cfg)
    assert st == bcs.BCS_OK, res
    assert true_rel(ref, system["b"], x) <= 1e-8
    if precision == bcs.BCS_PREC_FP64:
        assert abs(res["iters"] - ores["iters"]) <= 1, (res["iters"], ores["iters"])


@pytest.mark.parametrize("kw", [dict(), dict(precision=bcs.BCS_PREC_FP64), dict(precision=bcs.BCS_PREC_BF16),
                                dict(smoother=bcs.BCS_SMOOTH_DILU), dict(solver=bcs.BCS_BICGSTAB),
                                dict(pmode=bcs.BCS_P_SMOOTHED), dict(cycle_graph=0)],
                         ids=["fp32", "fp64", "bf16", "dilu", "bicgstab", "smoothed-P", "no-graph"])
def test_dependent_launch_identical(kw):
    """The V-cycle's kernels as programmatic dependent launches (each may be
    scheduled while its predecessor finishes and waits for its results):
    the same solve, bit for bit, as with ordinary launches."""
    system = synth.pressure(14, seed=3)
    out = []
    for dep in (0, 1):
        x, st, res = gpu_solve(system, dependent_launch=dep, **kw)
        assert st == bcs.BCS_OK, res
        out.append((x, res["iters"]))
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][0], out[1][0])


def test_x0_zero_ignores_x():
    """cfg.x0_zero: the solve starts from x = 0 whatever x holds on entry,
    for device and host memory and in a batched solve: the same result as a
    solve from an explicit zero vector."""
    system = synth.density(10, seed=6)
    junk = np.random.default_rng(5).standard_normal(system["b"].shape) * 1e3
    ref, st, res_ref = gpu_solve(system)
    assert st == bcs.BCS_OK
    for device in (True, False):
        x, st, res = gpu_solve(system, x0=junk, device=device, x0_zero=1)
        assert st == bcs.BCS_OK and res["iters"] == res_ref["iters"]
        assert np.array_equal(x, ref)
    with bcs.Solver(5, x0_zero=1) as s1, bcs.Solver(5, x0_zero=1) as s2:
        for s in (s1, s2):
            s.load(system, device=DEV)
        bs = [torch.from_numpy(system["b"]).to(DEV) for _ in range(2)]
        xs = [torch.from_numpy(junk).to(DEV) for _ in range(2)]
        xs, st, res = bcs.solve_batch([s1, s2], bs, xs)
        assert st == bcs.BCS_OK
        for x, r in zip(xs, res):
            assert r["status"] == bcs.BCS_OK and r["iters"] == res_ref["iters"]
            assert np.array_equal(x.cpu().numpy(), ref)


@pytest.mark.parametrize("solver", [bcs.BCS_FGMRES, bcs.BCS_BICGSTAB])
def test_resetup_keeps_graphs_identical(solver):
    """Values-only resetups rewrite the hierarchy in place, so the captured
    cycle and Krylov graphs are replayed across them: every solve of a
    resetup sequence equals the one of a solver without graphs bit for bit."""
    system = synth.pressure(12, seed=4)
    rng = [np.random.default_rng(17), np.random.default_rng(17)]
    out = {}
    for graph in (0, 1):
        xs = []
        sysg = system
        with bcs.Solver(4, solver=solver, cycle_graph=graph) as s:
            s.load(sysg, device=DEV)
            b = torch.from_numpy(sysg["b"]).to(DEV)
            for it in range(4):
                x, st, res = s.solve(b)
                assert st == bcs.BCS_OK
                xs.append((x.cpu().numpy(), res["iters"]))
                sysg = synth.perturb(sysg, rng[graph], 0.05)
                s.set_values(*(torch.from_numpy(sysg[k]).to(DEV) for k in ("diag", "upper", "lower")))
        out[graph] = xs
    for (x0, i0), (x1, i1) in zip(out[0], out[1]):
        assert i0 == i1 and np.array_equal(x0, x1)
