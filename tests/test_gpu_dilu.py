"""GPU parity of the multicolour block DILU smoother (Sec. 4): colourings and
FP64 factors E_i^-1 bit-exact with the CPU reference at every level (full
setup and values-only resetup); the V-cycle with DILU smoothing at 1e-12 in
FP64 and within FP32 / BF16 storage tolerance; solves to 1e-8 recomputed on
the CPU; the graph-replayed DILU cycle identical to kernel-by-kernel."""
import numpy as np
import pytest

import oracle
from paper_2403_07882_b300 import bcs, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
DILU = bcs.BCS_SMOOTH_DILU

CASES = [
    ("density 12^3", lambda: synth.density(12, seed=0), {}),
    ("density 9x7x5 smoothed", lambda: synth.density(9, 7, 5, seed=3), dict(pmode=0)),
    ("pressure 10^3", lambda: synth.pressure(10, seed=1), {}),
    ("knn 10^3", lambda: synth.knn(10, seed=2), {}),
    ("random n=3", lambda: synth.random_graph(400, 1500, 3, seed=5), dict(coarse_size=8)),
    ("density 24^3", lambda: synth.density(24, seed=4), {}),
]


def ocfg(**kw):
    return oracle.config(smoother=1, **{k: v for k, v in kw.items() if k != "precision"})


def compare_dilu(s, amg):
    assert s.levels == amg.levels
    for l in range(amg.levels):
        nc, col, einv = s.dilu(l)
        nr, col_r, einv_r = amg.dilu(l)
        assert nc == nr, l
        if nc > 0:
            assert np.array_equal(col, col_r), l
            assert np.array_equal(einv, einv_r), l


@pytest.mark.parametrize("name,gen,kw", CASES, ids=[c[0] for c in CASES])
def test_dilu_setup_and_resetup_bit_exact(name, gen, kw):
    system = gen()
    amg = oracle.Amg(oracle.ldu_to_bsr(system), ocfg(**kw))
    assert amg.status == 0
    with bcs.Solver(system["n"], precision=bcs.BCS_PREC_FP64, smoother=DILU, **kw) as s:
        s.load(system, device=DEV)
        compare_dilu(s, amg)
        system = synth.perturb(system, np.random.default_rng(4), 0.02)
        assert amg.resetup(oracle.ldu_to_bsr(system)["val"]) == 0
        s.set_values(*(torch.from_numpy(system[k]).to(DEV) for k in ("diag", "upper", "lower")))
        compare_dilu(s, amg)


@pytest.mark.parametrize("name,gen,kw", CASES, ids=[c[0] for c in CASES])
def test_dilu_vcycle_parity(name, gen, kw):
    system = gen()
    amg = oracle.Amg(oracle.ldu_to_bsr(system), ocfg(**kw))
    v = np.random.default_rng(6).standard_normal(system["b"].shape)
    z_ref = amg.vcycle(v)
    for prec, tol in ((bcs.BCS_PREC_FP64, None), (bcs.BCS_PREC_FP32, 2e-5), (bcs.BCS_PREC_BF16, 5e-2)):
        with bcs.Solver(system["n"], precision=prec, smoother=DILU, **kw) as s:
            s.load(system, device=DEV)
            z = s.precond(torch.from_numpy(v).to(DEV)).cpu().numpy()
        if tol is None:
            assert np.abs(z - z_ref).max() <= 1e-12 * np.abs(z_ref).max(), name
        else:
            assert np.linalg.norm(z - z_ref) <= tol * np.linalg.norm(z_ref), (name, prec)


@pytest.mark.parametrize("solver", [bcs.BCS_FGMRES, bcs.BCS_BICGSTAB], ids=["fgmres", "bicgstab"])
@pytest.mark.parametrize("gen", [lambda: synth.density(16, seed=0), lambda: synth.pressure(16, seed=1),
                                 lambda: synth.knn(14, seed=3)], ids=["density16", "pressure16", "knn14"])
def test_dilu_solves(gen, solver):
    system = gen()
    ref = oracle.ldu_to_bsr(system)
    its = {}
    for sm in (bcs.BCS_SMOOTH_JACOBI, DILU):
        with bcs.Solver(system["n"], solver=solver, smoother=sm) as s:
            s.load(system, device=DEV)
            x, st, res = s.solve(torch.from_numpy(system["b"]).to(DEV))
            assert st == bcs.BCS_OK, res
            xh = x.cpu().numpy()
        r = system["b"] - oracle.spmv(ref, xh)
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(system["b"])
        its[sm] = res["iters"]
    assert its[DILU] <= its[bcs.BCS_SMOOTH_JACOBI]


def test_dilu_graph_cycle_identical():
    system = synth.density(12, 10, 9, seed=7)
    v = np.random.default_rng(3).standard_normal(system["b"].shape)
    out = {}
    for graph in (0, 1):
        with bcs.Solver(5, smoother=DILU, cycle_graph=graph) as s:
            s.load(system, device=DEV)
            vt = torch.from_numpy(v).to(DEV)
            out[graph] = (s.precond(vt).cpu().numpy(), s.precond(vt).cpu().numpy())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[1][0], out[1][1])


CLUSTER_CASES = [
    ("density 16^3 DILU fp32", lambda: synth.density(16, seed=0), dict(smoother=DILU)),
    ("density 16^3 DILU bf16", lambda: synth.density(16, seed=0), dict(smoother=DILU, precision=bcs.BCS_PREC_BF16)),
    ("pressure 20^3 DILU, tpr layout", lambda: synth.pressure(20, seed=2), dict(smoother=DILU, slice_layout=1)),
    ("knn 14 DILU", lambda: synth.knn(14, seed=3), dict(smoother=DILU)),
    ("density 12^3 SGS smoother", lambda: synth.density(12, seed=4), dict(smoother=bcs.BCS_SMOOTH_SGS)),
    ("density 12^3 SGS preconditioner", lambda: synth.density(12, seed=4),
     dict(precond=bcs.BCS_PC_SGS, maxiter=5000)),
]


@pytest.mark.parametrize("name,gen,kw", CLUSTER_CASES, ids=[c[0] for c in CLUSTER_CASES])
def test_dilu_cluster_step_identical(name, gen, kw):
    """Levels below dilu_cluster_rows run a DILU / SGS step (residual and
    every colour of both sweeps) as one thread-block-cluster launch: the same
    solve as with one launch per colour (dilu_cluster_rows = 0), bit for
    bit, with and without the graph-replayed cycle."""
    system = gen()
    b = torch.from_numpy(system["b"]).to(DEV)
    out = {}
    for rows, graph in ((0, 1), (1 << 30, 1), (1 << 30, 0)):
        with bcs.Solver(system["n"], dilu_cluster_rows=rows, cycle_graph=graph, **kw) as s:
            s.load(system, device=DEV)
            x, st, res = s.solve(b)
            assert st == bcs.BCS_OK, res
            out[(rows, graph)] = (x.cpu().numpy(), res["iters"], s.stats()["kinds"]["jacobi_sweep"]["launches"])
    ref = out[(0, 1)]
    for key, (x, it, n) in out.items():
        assert it == ref[1], key
        assert np.array_equal(x, ref[0]), key
        if key[0]:
            assert 0 < n < ref[2], (key, n, ref[2])  # one launch per step instead of 2 x colours
