"""The device-resident Krylov loops against the host-driven ones. FGMRES:
the Arnoldi step replayed in a CUDA graph WHILE node, Givens rotations,
least-squares update and the stop test in FP64 device kernels, one host
read per restart cycle. BiCGStab: the iteration replayed the same way, its
scalars and tests in kernels, the host acting only on events. Both give the
host loops' iterates bit for bit, the same iteration and restart counts,
fewer host synchronisations, and the true residual 1e-8 recomputed by the
oracle (GMRES of Saad and Schultz, Sec. 2; Sec. 2.3's GMRES and BiCGStab)."""
import numpy as np
import pytest

import oracle
from paper_2403_07882_b300 import bcs, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

CASES = [
    ("density 16^3 fp32", lambda: synth.density(16, seed=0), dict()),
    ("density 16^3 bf16", lambda: synth.density(16, seed=0), dict(precision=bcs.BCS_PREC_BF16)),
    ("density 12^3 fp64", lambda: synth.density(12, seed=2), dict(precision=bcs.BCS_PREC_FP64)),
    ("pressure 12^3 m=5 fp32", lambda: synth.pressure(12, seed=1), dict(restart=5)),
    ("pressure 12^3 m=3 fp64", lambda: synth.pressure(12, seed=1), dict(restart=3, precision=bcs.BCS_PREC_FP64)),
    ("density 12^3 dilu", lambda: synth.density(12, seed=3), dict(smoother=bcs.BCS_SMOOTH_DILU)),
    ("density 12^3 sgs preconditioner", lambda: synth.density(12, seed=3), dict(precond=bcs.BCS_PC_SGS)),
    ("density 10^3 sgs fp64", lambda: synth.density(10, seed=4),
     dict(precond=bcs.BCS_PC_SGS, precision=bcs.BCS_PREC_FP64)),
    ("knn 12 maxiter 3", lambda: synth.knn(12, seed=5), dict(maxiter=3)),
    ("bicgstab density 16^3 fp32", lambda: synth.density(16, seed=0), dict(solver=bcs.BCS_BICGSTAB)),
    ("bicgstab pressure 14^3 fp32", lambda: synth.pressure(14, seed=1), dict(solver=bcs.BCS_BICGSTAB)),
    ("bicgstab pressure 12^3 fp64", lambda: synth.pressure(12, seed=3),
     dict(solver=bcs.BCS_BICGSTAB, precision=bcs.BCS_PREC_FP64)),
    ("bicgstab density 12^3 bf16", lambda: synth.density(12, seed=2),
     dict(solver=bcs.BCS_BICGSTAB, precision=bcs.BCS_PREC_BF16)),
    ("bicgstab density 10^3 sgs", lambda: synth.density(10, seed=4),
     dict(solver=bcs.BCS_BICGSTAB, precond=bcs.BCS_PC_SGS)),
    ("bicgstab knn 12 maxiter 2", lambda: synth.knn(12, seed=5), dict(solver=bcs.BCS_BICGSTAB, maxiter=2)),
]


def run(system, graph, **cfg):
    with bcs.Solver(system["n"], cycle_graph=graph, **cfg) as s:
        s.load(system, device=DEV)
        b = torch.from_numpy(system["b"]).to(DEV)
        s.reset_stats()
        x, st, res = s.solve(b)
        launches = s.stats()["launches"]
        # a second solve replays the captured loop
        x2, st2, res2 = s.solve(b)
        assert st2 == st and torch.equal(x, x2) and res2["iters"] == res["iters"]
    return x.cpu().numpy(), st, res, launches


@pytest.mark.parametrize("name,gen,cfg", CASES, ids=[c[0] for c in CASES])
def test_device_cycle_equals_host_loop(name, gen, cfg):
    system = gen()
    xh, sth, rh, lh = run(system, 0, **cfg)
    xd, std, rd, ld = run(system, 1, **cfg)
    assert std == sth
    assert rd["iters"] == rh["iters"] and rd["restarts"] == rh["restarts"]
    assert np.array_equal(xd, xh)
    assert rd["rel_res_final"] == rh["rel_res_final"]
    if std == bcs.BCS_OK:
        ref = oracle.ldu_to_bsr(system)
        r = system["b"] - oracle.spmv(ref, xd)
        assert np.linalg.norm(r) / np.linalg.norm(system["b"]) <= 1e-8
    else:
        assert std == bcs.BCS_NOT_CONVERGED and rd["iters"] == cfg.get("maxiter")
    # the device loops read the device once per restart cycle (FGMRES) or per
    # event (BiCGStab), the host loops once or more per iteration
    assert rd["host_syncs"] < rh["host_syncs"]
    print(f"{name}: iters={rd['iters']} restarts={rd['restarts']} launches host={lh} device={ld} "
          f"host syncs {rh['host_syncs']} -> {rd['host_syncs']}")


def test_device_cycle_after_resetup_and_restart_change():
    """The captured loop follows a values-only resetup (new hierarchy values,
    same buffers) and a change of the restart length (new buffers)."""
    system = synth.density(12, seed=6)
    rng = np.random.default_rng(2)
    out = {}
    for graph in (0, 1):
        with bcs.Solver(5, cycle_graph=graph) as s:
            s.load(system, device=DEV)
            b = torch.from_numpy(system["b"]).to(DEV)
            xs = [s.solve(b)[0].cpu().numpy()]
            sys2 = synth.perturb(system, rng if graph == 0 else np.random.default_rng(2), 0.02)
            s.set_values(*(torch.from_numpy(sys2[k]).to(DEV) for k in ("diag", "upper", "lower")))
            xs.append(s.solve(b)[0].cpu().numpy())
            s.set_config(restart=4)
            x, st, res = s.solve(b)
            assert st == bcs.BCS_OK and res["restarts"] >= 1
            xs.append(x.cpu().numpy())
            out[graph] = xs
    for a, c in zip(out[0], out[1]):
        assert np.array_equal(a, c)
