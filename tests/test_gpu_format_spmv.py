"""GPU parity: LDU -> block-CSR conversion (bit-exact) and FP64 BSR SpMV
(1e-12 relative to (|A| |x|)_i) against the CPU reference, through the C ABI.
"""
import numpy as np
import pytest

import oracle
from paper_2403_07882_b300 import bcs, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def systems():
    return [
        ("density 2x2x2", synth.density(2, 2, 2, seed=5)),
        ("density 3x2x1", synth.density(3, 2, 1, seed=6)),
        ("density 16^3 (c1)", synth.density(16, seed=0)),
        ("pressure 12^3", synth.pressure(12, seed=1)),
        ("random n=1", synth.random_graph(40, 90, 1, seed=1)),
        ("random n=3", synth.random_graph(50, 120, 3, seed=2)),
        ("random n=7", synth.random_graph(30, 60, 7, seed=3)),
        ("random n=8", synth.random_graph(33, 70, 8, seed=4)),
    ]


def spmv_ok(y, y_ref, absA_absx, tol=1e-12):
    return np.all(np.abs(y - y_ref) <= tol * absA_absx + 1e-300)


def abs_product(ref, x):
    absref = dict(ref)
    absref["val"] = np.abs(ref["val"])
    return oracle.spmv(absref, np.abs(x))


@pytest.mark.parametrize("name,system", systems(), ids=[s[0] for s in systems()])
@pytest.mark.parametrize("where", ["device", "host"])
def test_bsr_bit_exact(name, system, where):
    ref = oracle.ldu_to_bsr(system)
    with bcs.Solver(system["n"]) as s:
        s.load(system, device=DEV if where == "device" else None)
        got = s.bsr()
    for key in ("row_ptr", "col", "pos_diag", "pos_up", "pos_lo"):
        assert np.array_equal(got[key], ref[key]), key
    assert np.array_equal(got["val"], ref["val"])
    # round trip LDU -> BSR -> LDU
    assert np.array_equal(got["val"][got["pos_up"]], system["upper"])
    assert np.array_equal(got["val"][got["pos_lo"]], system["lower"])
    assert np.array_equal(got["val"][got["pos_diag"]], system["diag"])


def test_reversed_faces_accepted():
    system = synth.random_graph(20, 40, 2, seed=9)
    flip = np.arange(system["n_faces"]) % 3 == 0
    o, m = system["owner"].copy(), system["neighbour"].copy()
    system["owner"] = np.where(flip, m, o).astype(np.int32)
    system["neighbour"] = np.where(flip, o, m).astype(np.int32)
    ref = oracle.ldu_to_bsr(system)
    with bcs.Solver(2) as s:
        s.load(system, device=DEV)
        got = s.bsr()
    assert np.array_equal(got["col"], ref["col"]) and np.array_equal(got["val"], ref["val"])


@pytest.mark.parametrize("owner,neighbour,C", [
    ([0, 1], [1, 3], 3), ([0, 1], [1, 1], 3), ([0, 1, 1], [1, 2, 0], 3), ([0, 0], [1, 1], 2), ([-1], [0], 2)])
def test_structure_rejects(owner, neighbour, C):
    with bcs.Solver(2) as s:
        with pytest.raises(bcs.BcsError) as e:
            s.set_structure(C, torch.tensor(owner, dtype=torch.int32, device=DEV),
                            torch.tensor(neighbour, dtype=torch.int32, device=DEV))
        assert e.value.status == bcs.BCS_EINVAL
        with pytest.raises(bcs.BcsError) as e:   # no structure kept
            s.set_values(np.ones((C, 2, 2)), np.ones((len(owner), 2, 2)), np.ones((len(owner), 2, 2)))
        assert e.value.status == bcs.BCS_ESTATE


def test_single_cell_no_faces():
    rng = np.random.default_rng(0)
    D = rng.standard_normal((1, 4, 4)) + 4 * np.eye(4)
    system = dict(n_cells=1, n_faces=0, n=4, owner=np.zeros(0, np.int32), neighbour=np.zeros(0, np.int32),
                  diag=D, upper=np.zeros((0, 4, 4)), lower=np.zeros((0, 4, 4)), b=rng.standard_normal((1, 4)))
    with bcs.Solver(4) as s:
        s.load(system)
        x = rng.standard_normal((1, 4))
        assert np.allclose(s.spmv(x)[0], D[0] @ x[0], rtol=1e-15, atol=1e-15)
        xs, st, res = s.solve(system["b"])
        assert st == bcs.BCS_OK
        assert np.allclose(D[0] @ xs[0], system["b"][0], rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("name,system", systems(), ids=[s[0] for s in systems()])
def test_spmv_fp64_parity(name, system):
    ref = oracle.ldu_to_bsr(system)
    x = np.random.default_rng(7).standard_normal(system["b"].shape)
    with bcs.Solver(system["n"]) as s:
        s.load(system, device=DEV)
        y = s.spmv(torch.from_numpy(x).to(DEV)).cpu().numpy()
        y_host = s.spmv(x)
    y_ref = oracle.spmv(ref, x)
    scale = abs_product(ref, x)
    assert spmv_ok(y, y_ref, scale)
    assert np.array_equal(y, y_host)


def test_spmv_identity_blocks_exact():
    system = synth.density(5, 4, 3, seed=1)
    system["diag"][:] = np.eye(5)
    system["upper"][:] = 0.0
    system["lower"][:] = 0.0
    with bcs.Solver(5) as s:
        s.load(system)
        x = np.random.default_rng(0).standard_normal(system["b"].shape)
        assert np.array_equal(s.spmv(x), x)


def test_full_size_128cube_conversion_and_spmv():
    """The 128^3 5x5 density-based workload (2.1 M cells, 14.6 M blocks) in
    the benchmark's launch configuration: structure maps exact, sampled
    values exact, SpMV against the CPU reference at 1e-12."""
    system = synth.density(128, seed=2)
    ref = oracle.ldu_to_bsr(system)
    with bcs.Solver(5, precond=bcs.BCS_PC_NONE) as s:
        s.load(system, device=DEV)
        got = s.bsr(values=False)
        for key in ("row_ptr", "col", "pos_diag", "pos_up", "pos_lo"):
            assert np.array_equal(got[key], ref[key]), key
        x = np.random.default_rng(3).standard_normal(system["b"].shape)
        y = s.spmv(torch.from_numpy(x).to(DEV)).cpu().numpy()
    y_ref = oracle.spmv(ref, x)
    assert spmv_ok(y, y_ref, abs_product(ref, x))
