"""Unstructured workload (config 4 generator at a reduced size): jittered
lattice points linked to k-nearest neighbours (k ~ U{4..12}, symmetrised),
so rows have irregular lengths. Setup bit-exact with the CPU reference, FP64
SpMV parity, and the Alg. 1 sequence of values-only resetups (2 % value
perturbation per nonlinear iteration) each solved to 1e-8."""
import numpy as np
import pytest

import oracle
from paper_2403_07882_b300 import bcs, synth
from test_gpu_amg import compare_hierarchy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def knn_system():
    return synth.knn(20, seed=3)


def test_knn_setup_bit_exact_and_spmv(knn_system):
    system = knn_system
    ref = oracle.ldu_to_bsr(system)
    amg = oracle.Amg(ref, oracle.config())
    with bcs.Solver(5, precision=bcs.BCS_PREC_FP64) as s:
        s.load(system, device=DEV)
        compare_hierarchy(s, amg, 5, 1)
        x = np.random.default_rng(1).standard_normal(system["b"].shape)
        y = s.spmv(torch.from_numpy(x).to(DEV)).cpu().numpy()
    absref = dict(ref)
    absref["val"] = np.abs(ref["val"])
    scale = oracle.spmv(absref, np.abs(x))
    assert np.all(np.abs(y - oracle.spmv(ref, x)) <= 1e-12 * scale)


def test_knn_resetup_sequence(knn_system):
    system = knn_system
    rng = np.random.default_rng(7)
    amg = oracle.Amg(oracle.ldu_to_bsr(system), oracle.config())
    with bcs.Solver(5) as s:
        s.load(system, device=DEV)
        b = torch.from_numpy(system["b"]).to(DEV)
        for it in range(10):
            system = synth.perturb(system, rng, 0.02)
            ref = oracle.ldu_to_bsr(system)
            assert amg.resetup(ref["val"]) == 0
            s.set_values(*(torch.from_numpy(system[k]).to(DEV) for k in ("diag", "upper", "lower")))
            x, st, res = s.solve(b)
            assert st == bcs.BCS_OK
            xh = x.cpu().numpy()
            r = system["b"] - oracle.spmv(ref, xh)
            assert np.linalg.norm(r) / np.linalg.norm(system["b"]) <= 1e-8
        # the resetup hierarchy is the reference's resetup hierarchy
        g = s.level(1)
        assert np.array_equal(g["val"], amg.A(1)["val"])
