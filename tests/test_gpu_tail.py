"""The coarse tail of the V-cycle (every level of at most tail_rows block
rows, run as one thread-block-cluster launch per cycle with cluster
barriers between its phases) against the same cycle launched kernel by
kernel: identical preconditioner outputs and solves, bit for bit, for FP32
and BF16 storage, with the tail starting at the fine level (the whole cycle
in one launch) or deeper; and the FP32 cycle within its tolerance of the
FP64 oracle (the aggregation AMG V-cycle of Sec. 2.3)."""
import numpy as np
import pytest

import oracle
from paper_2403_07882_b300 import bcs, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

CASES = [
    ("density 16^3 whole cycle", lambda: synth.density(16, seed=0), dict(tail_rows=8192)),
    ("density 24^3 tail below fine", lambda: synth.density(24, seed=1), dict(tail_rows=4000)),
    ("pressure 20^3", lambda: synth.pressure(20, seed=2), dict(tail_rows=2000)),
    ("knn 16 uneven rows", lambda: synth.knn(16, seed=5), dict(tail_rows=1500)),
    ("random n=3 tiny levels", lambda: synth.random_graph(3000, 12000, 3, seed=3), dict(tail_rows=700)),
    ("density 12^3 coarse sweeps", lambda: synth.density(12, seed=4), dict(tail_rows=8192, coarse_dense_max=1)),
    ("density 12^3 nu 1+3", lambda: synth.density(12, seed=4), dict(tail_rows=8192, nu1=1, nu2=3)),
    ("density 12^3 nu 0+2", lambda: synth.density(12, seed=4), dict(tail_rows=8192, nu1=0, nu2=2)),
]


def run(system, precision, graph, **kw):
    with bcs.Solver(system["n"], precision=precision, cycle_graph=graph, **kw) as s:
        s.load(system, device=DEV)
        v = torch.from_numpy(np.random.default_rng(7).standard_normal(system["b"].shape)).to(DEV)
        s.reset_stats()
        z = s.precond(v).cpu().numpy()
        launches = s.stats()["launches"]
        x, st, res = s.solve(torch.from_numpy(system["b"]).to(DEV))
        assert st == bcs.BCS_OK, res
        return z, x.cpu().numpy(), res["iters"], launches


@pytest.mark.parametrize("precision", [bcs.BCS_PREC_FP32, bcs.BCS_PREC_BF16])
@pytest.mark.parametrize("name,gen,kw", CASES, ids=[c[0] for c in CASES])
def test_tail_equals_kernel_by_kernel(name, gen, kw, precision):
    system = gen()
    z0, x0, it0, l0 = run(system, precision, 0, **{**kw, "tail_rows": 0})
    z1, x1, it1, l1 = run(system, precision, 0, **kw)
    z2, x2, it2, l2 = run(system, precision, 1, **kw)   # graph replay of the cycle with the tail
    assert np.array_equal(z0, z1) and np.array_equal(z0, z2)
    assert np.array_equal(x0, x1) and np.array_equal(x0, x2) and it0 == it1 == it2
    assert l1 < l0
    if precision == bcs.BCS_PREC_FP32:
        okw = {k: v for k, v in kw.items() if k != "tail_rows"}
        amg = oracle.Amg(oracle.ldu_to_bsr(system), oracle.config(**okw))
        v = np.random.default_rng(7).standard_normal(system["b"].shape)
        z_ref = amg.vcycle(v)
        assert np.linalg.norm(z1 - z_ref) <= 2e-5 * np.linalg.norm(z_ref)
    print(f"{name}: launches per cycle {l0} -> {l1}")
