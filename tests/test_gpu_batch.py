"""Batched solves (bcs_solve_batch): several systems of uneven size and
hierarchy depth solved together, their FGMRES steps (Sec. 2; Sec. 2.3's
GMRES with aggregation AMG) in lockstep with one launch per V-cycle phase
and level for the whole batch. Every system's solution, iteration and
restart counts equal those of solving it alone, bit for bit, for FP32 and
BF16 storage, with restarts, a system needing no iteration, host and device
arrays; incompatible solvers are refused."""
import numpy as np
import pytest

import oracle
from paper_2403_07882_b300 import bcs, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def systems():
    return [synth.density(14, seed=1), synth.density(9, 7, 5, seed=2), synth.knn(9, seed=3),
            synth.random_graph(2000, 7000, 5, seed=4), synth.density(22, 18, 16, seed=5), synth.density(3, seed=6)]


def alone(system, **cfg):
    with bcs.Solver(system["n"], **cfg) as s:
        s.load(system, device=DEV)
        x, st, res = s.solve(torch.from_numpy(system["b"]).to(DEV))
        return x.cpu().numpy(), st, res


@pytest.mark.parametrize("cfg", [dict(), dict(precision=bcs.BCS_PREC_BF16), dict(restart=4)],
                         ids=["fp32", "bf16", "restart4"])
def test_batch_equals_alone(cfg):
    sys_ = systems()
    ref = [alone(s, **cfg) for s in sys_]
    solvers = [bcs.Solver(s["n"], **cfg) for s in sys_]
    try:
        for s, sy in zip(solvers, sys_):
            s.load(sy, device=DEV)
        bs = [torch.from_numpy(sy["b"]).to(DEV) for sy in sys_]
        xs, st, res = bcs.solve_batch(solvers, bs)
        assert st == bcs.BCS_OK
        levels = set()
        for i, sy in enumerate(sys_):
            x_ref, st_ref, r_ref = ref[i]
            assert st_ref == bcs.BCS_OK and res[i]["status"] == bcs.BCS_OK
            assert res[i]["iters"] == r_ref["iters"] and res[i]["restarts"] == r_ref["restarts"], i
            assert np.array_equal(xs[i].cpu().numpy(), x_ref), i
            assert res[i]["rel_res_final"] == r_ref["rel_res_final"]
            levels.add(res[i]["levels"])
            b = sy["b"]
            r = b - oracle.spmv(oracle.ldu_to_bsr(sy), xs[i].cpu().numpy())
            assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-8
        assert len(levels) >= 3   # uneven hierarchy depths in one batch
        if cfg.get("restart") == 4:
            assert max(r["restarts"] for r in res) >= 1
    finally:
        for s in solvers:
            s.close()


def test_batch_host_arrays_zero_rhs_and_warm_start():
    sys_ = systems()[:4]
    sys_[1] = dict(sys_[1])
    sys_[1]["b"] = np.zeros_like(sys_[1]["b"])          # b = 0: x = 0, no iteration
    ref = [alone(s) for s in sys_]
    solvers = [bcs.Solver(s["n"]) for s in sys_]
    try:
        for s, sy in zip(solvers, sys_):
            s.load(sy, device=DEV)
        xs = [np.ones_like(sy["b"]) for sy in sys_]
        xs[2] = ref[2][0].copy()                          # already converged: no iteration
        xs[0] = np.zeros_like(sys_[0]["b"])
        xs[3] = np.zeros_like(sys_[3]["b"])
        xs, st, res = bcs.solve_batch(solvers, [sy["b"] for sy in sys_], xs)
        assert st == bcs.BCS_OK
        assert np.all(xs[1] == 0) and res[1]["iters"] == 0
        assert res[2]["iters"] <= 1
        for i in (0, 3):
            assert np.array_equal(xs[i], ref[i][0]) and res[i]["iters"] == ref[i][2]["iters"]
    finally:
        for s in solvers:
            s.close()


def test_batch_refuses_incompatible_solvers():
    a, b = synth.density(6, seed=1), synth.pressure(6, seed=2)
    with bcs.Solver(5) as s1, bcs.Solver(4) as s2, bcs.Solver(5, smoother=bcs.BCS_SMOOTH_DILU) as s3:
        s1.load(a, device=DEV)
        s2.load(b, device=DEV)
        s3.load(a, device=DEV)
        for other, sy in ((s2, b), (s3, a)):
            with pytest.raises(bcs.BcsError) as e:
                bcs.solve_batch([s1, other], [torch.from_numpy(a["b"]).to(DEV), torch.from_numpy(sy["b"]).to(DEV)])
            assert e.value.status == bcs.BCS_EINVAL
        with bcs.Solver(5) as s4:
            s4.set_structure(a["n_cells"], a["owner"], a["neighbour"])
            with pytest.raises(bcs.BcsError) as e:
                bcs.solve_batch([s1, s4], [torch.from_numpy(a["b"]).to(DEV)] * 2)
            assert e.value.status == bcs.BCS_ESTATE
