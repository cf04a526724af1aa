"""GPU parity of the AMG setup (aggregates, Galerkin operators, block and
coarse inverses, smoothed prolongation: bit-exact with the FP64 CPU
reference) and of the V-cycle (1e-12 in FP64; FP32/BF16 storage within a
tolerance derived from the storage precision)."""
import numpy as np
import pytest

import oracle
from paper_2403_07882_b300 import bcs, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

CASES = [
    ("density 16^3", lambda: synth.density(16, seed=0), {}),
    ("density 10x7x5 smoothed", lambda: synth.density(10, 7, 5, seed=3), dict(pmode=0)),
    ("pressure 12^3", lambda: synth.pressure(12, seed=1), {}),
    ("pressure 9^3 smoothed", lambda: synth.pressure(9, seed=2), dict(pmode=0)),
    ("random n=3 one pass", lambda: synth.random_graph(300, 900, 3, seed=5), dict(agg_passes=1, coarse_size=8)),
    ("random n=2 three passes", lambda: synth.random_graph(400, 1000, 2, seed=6), dict(agg_passes=3, coarse_size=4)),
    # coarsest level of 81 rows x 4 = 324 unknowns (above 96): the dense inverse
    # runs on a cooperative grid (the cases above take the shared-memory form)
    ("pressure 12^3 large dense coarse", lambda: synth.pressure(12, seed=1), dict(coarse_size=200)),
]


def oracle_cfg(**kw):
    return oracle.config(**{k: v for k, v in kw.items() if k != "precision"})


def compare_hierarchy(s, amg, n, pmode):
    assert s.levels == amg.levels
    for l in range(amg.levels):
        g = s.level(l)
        A = amg.A(l)
        assert np.array_equal(g["row_ptr"], A["row_ptr"]), l
        assert np.array_equal(g["col"], A["col"]), l
        assert np.array_equal(g["val"], A["val"]), l
        assert np.array_equal(g["dinv"], amg.dinv(l)), l
        info = amg.info(l)
        assert g["coarse_kind"] == info["coarse_kind"]
        if info["coarse_kind"] < 0:
            P = amg.P(l)
            assert np.array_equal(g["agg"], P["agg"]), l
            if pmode == 0:
                gp = s.prolongation(l)
                assert gp["omega"] == P["omega"]
                assert np.array_equal(gp["row_ptr"], P["row_ptr"]) and np.array_equal(gp["col"], P["col"])
                assert np.array_equal(gp["val"], P["val"])
    if amg.info(amg.levels - 1)["coarse_kind"] == 0:
        assert np.array_equal(s.coarse_inverse(), amg.coarse_inverse())


@pytest.mark.parametrize("name,gen,kw", CASES, ids=[c[0] for c in CASES])
def test_setup_bit_exact(name, gen, kw):
    system = gen()
    ref = oracle.ldu_to_bsr(system)
    amg = oracle.Amg(ref, oracle_cfg(**kw))
    assert amg.status == 0
    with bcs.Solver(system["n"], precision=bcs.BCS_PREC_FP64, **kw) as s:
        s.load(system, device=DEV)
        compare_hierarchy(s, amg, system["n"], kw.get("pmode", 1))


@pytest.mark.parametrize("name,gen,kw", CASES, ids=[c[0] for c in CASES])
def test_resetup_bit_exact(name, gen, kw):
    system = gen()
    ref = oracle.ldu_to_bsr(system)
    amg = oracle.Amg(ref, oracle_cfg(**kw))
    rng = np.random.default_rng(11)
    with bcs.Solver(system["n"], precision=bcs.BCS_PREC_FP64, **kw) as s:
        s.load(system, device=DEV)
        for _ in range(2):
            system = synth.perturb(system, rng, 0.02)
            new = oracle.ldu_to_bsr(system)
            assert amg.resetup(new["val"]) == 0
            s.set_values(*(torch.from_numpy(system[k]).to(DEV) for k in ("diag", "upper", "lower")))
            compare_hierarchy(s, amg, system["n"], kw.get("pmode", 1))


@pytest.mark.parametrize("name,gen,kw", CASES, ids=[c[0] for c in CASES])
def test_vcycle_fp64_parity(name, gen, kw):
    system = gen()
    ref = oracle.ldu_to_bsr(system)
    amg = oracle.Amg(ref, oracle_cfg(**kw))
    v = np.random.default_rng(4).standard_normal(system["b"].shape)
    z_ref = amg.vcycle(v)
    with bcs.Solver(system["n"], precision=bcs.BCS_PREC_FP64, **kw) as s:
        s.load(system, device=DEV)
        z = s.precond(torch.from_numpy(v).to(DEV)).cpu().numpy()
    assert np.abs(z - z_ref).max() <= 1e-12 * np.abs(z_ref).max()


@pytest.mark.parametrize("precision,tol", [(bcs.BCS_PREC_FP32, 2e-5), (bcs.BCS_PREC_BF16, 5e-2)])
@pytest.mark.parametrize("name,gen,kw", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_vcycle_low_precision(precision, tol, name, gen, kw):
    """FP32 storage/arithmetic: unit roundoff 6e-8 amplified by the cycle's
    few dozen operations and the operator norms gives a 2e-5 bound relative
    to ||z||; BF16 storage (roundoff 4e-3) perturbs the operator itself, so
    only a 5e-2 relative agreement is expected."""
    system = gen()
    ref = oracle.ldu_to_bsr(system)
    amg = oracle.Amg(ref, oracle_cfg(**kw))
    v = np.random.default_rng(5).standard_normal(system["b"].shape)
    z_ref = amg.vcycle(v)
    with bcs.Solver(system["n"], precision=precision, **kw) as s:
        s.load(system, device=DEV)
        z = s.precond(torch.from_numpy(v).to(DEV)).cpu().numpy()
    assert np.linalg.norm(z - z_ref) <= tol * np.linalg.norm(z_ref)


def test_singular_block_reported():
    system = synth.density(6, seed=6)
    system["diag"][4] = 0.0
    with bcs.Solver(5) as s:
        with pytest.raises(bcs.BcsError) as e:
            s.load(system, device=DEV)
        assert e.value.status == bcs.BCS_SINGULAR_BLOCK
        with pytest.raises(bcs.BcsError) as e:
            bcs.bcs_solve(s.h, system["b"], np.zeros_like(system["b"]))
        assert e.value.status == bcs.BCS_ESTATE


def test_determinism_two_setups():
    system = synth.pressure(16, seed=4)
    outs = []
    for _ in range(2):
        with bcs.Solver(4, precision=bcs.BCS_PREC_FP32) as s:
            s.load(system, device=DEV)
            v = torch.from_numpy(system["b"]).to(DEV)
            outs.append(s.precond(v).cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("gen", [lambda: synth.density(20, seed=1), lambda: synth.pressure(14, seed=2),
                                 lambda: synth.random_graph(3000, 12000, 3, seed=3), lambda: synth.knn(14, seed=5)])
def test_fp32_sliced_cycle_on_uneven_rows(gen):
    """The FP32 cycle with sliced storage agrees with the FP64 reference cycle
    to FP32 rounding on rows of uneven length (slice padding) for n = 3, 4, 5."""
    system = gen()
    ref = oracle.ldu_to_bsr(system)
    amg = oracle.Amg(ref, oracle.config())
    v = np.random.default_rng(9).standard_normal(system["b"].shape)
    z_ref = amg.vcycle(v)
    with bcs.Solver(system["n"], precision=bcs.BCS_PREC_FP32) as s:
        s.load(system, device=DEV)
        z = s.precond(torch.from_numpy(v).to(DEV)).cpu().numpy()
    assert np.linalg.norm(z - z_ref) <= 2e-5 * np.linalg.norm(z_ref)


@pytest.mark.parametrize("precision", [bcs.BCS_PREC_FP32, bcs.BCS_PREC_BF16])
@pytest.mark.parametrize("gen", [lambda: synth.density(20, seed=1), lambda: synth.pressure(18, seed=2),
                                 lambda: synth.knn(16, seed=5), lambda: synth.random_graph(5000, 20000, 3, seed=3)])
def test_slice_layouts_identical(gen, precision):
    """Both storage layouts of the low-precision cycle (one lane per scalar
    row; one thread per block row) run the same fma sequence per scalar row,
    so the preconditioner outputs are bit-identical; the tuned default equals
    both, and all agree with the FP64 reference cycle to storage precision."""
    system = gen()
    v = np.random.default_rng(12).standard_normal(system["b"].shape)
    outs = {}
    for layout in (0, 1, -1):
        with bcs.Solver(system["n"], precision=precision, slice_layout=layout) as s:
            s.load(system, device=DEV)
            outs[layout] = s.precond(torch.from_numpy(v).to(DEV)).cpu().numpy()
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[-1])
    amg = oracle.Amg(oracle.ldu_to_bsr(system), oracle.config())
    z_ref = amg.vcycle(v)
    tol = 2e-5 if precision == bcs.BCS_PREC_FP32 else 5e-2
    assert np.linalg.norm(outs[0] - z_ref) <= tol * np.linalg.norm(z_ref)


def tpr_fill_launches(s):
    return sum(t["launches"] for name, t in s.kernel_times().items() if name.startswith("(k_tpr_fill"))


@pytest.mark.parametrize("precision", [bcs.BCS_PREC_FP32, bcs.BCS_PREC_BF16])
@pytest.mark.parametrize("host", [False, True], ids=["device-values", "host-values"])
@pytest.mark.parametrize("cfg", [dict(), dict(smoother=bcs.BCS_SMOOTH_DILU), dict(precond=bcs.BCS_PC_SGS)],
                         ids=["amg-jacobi", "amg-dilu", "sgs"])
def test_gather_writes_fine_sliced_copy(precision, host, cfg):
    """The first setup of a structure fills the fine level's thread-per-row
    FP32 / BF16 copy and records each block's slot; at every values-only
    resetup the value gather writes the copy through those slots and the
    fill kernel skips that level. Same values give the same preconditioner
    bits; new values give those of the lane-per-row layout filled from the
    block-CSR values (bit for bit with block Jacobi, whose layouts share one
    fma order; within the storage precision with DILU / SGS sweeps)."""
    system = synth.density(20, seed=1)
    v = torch.from_numpy(np.random.default_rng(12).standard_normal(system["b"].shape)).to(DEV)
    dev = {k: torch.from_numpy(system[k]).to(DEV) for k in ("owner", "neighbour", "diag", "upper", "lower")}
    vals1 = [system[k] if host else dev[k] for k in ("diag", "upper", "lower")]
    vals2 = [vals1[0], 0.8 * vals1[1], 0.7 * vals1[2]]
    z, fills = {}, []
    for layout in (1, 0):
        with bcs.Solver(5, precision=precision, slice_layout=layout, profile=1, **cfg) as s:
            s.set_structure(system["n_cells"], dev["owner"], dev["neighbour"])
            for phase, vals in (("setup", vals1), ("resetup-same", vals1), ("resetup-new", vals2)):
                s.reset_stats()
                s.set_values(*vals)
                if layout == 1:
                    fills.append(tpr_fill_launches(s))
                z[layout, phase] = s.precond(v).cpu().numpy()
    assert fills[0] >= 1 and fills[1] == fills[2] == fills[0] - 1, fills
    assert np.array_equal(z[1, "resetup-same"], z[1, "setup"])
    new, ref = z[1, "resetup-new"], z[0, "resetup-new"]
    assert np.linalg.norm(new - z[1, "setup"]) > 1e-2 * np.linalg.norm(ref)  # the values did change
    if not cfg:
        assert np.array_equal(new, ref)
    else:
        tol = 1e-5 if precision == bcs.BCS_PREC_FP32 else 2e-2
        assert np.linalg.norm(new - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("precision", [bcs.BCS_PREC_FP32, bcs.BCS_PREC_BF16])
def test_graph_cycle_identical(precision):
    """The V-cycle replayed as a CUDA graph gives the same bits as the same
    cycle launched kernel by kernel, counts the same launches, and solves
    (FGMRES and BiCGStab) give identical iterates; a resetup drops and
    recaptures the graph."""
    system = synth.density(12, 10, 9, seed=7)
    v = np.random.default_rng(3).standard_normal(system["b"].shape)
    res = {}
    for graph in (0, 1):
        with bcs.Solver(5, precision=precision, cycle_graph=graph) as s:
            s.load(system, device=DEV)
            vt = torch.from_numpy(v).to(DEV)
            s.reset_stats()
            z1 = s.precond(vt).cpu().numpy()
            z2 = s.precond(vt).cpu().numpy()
            launches = s.stats()["launches"]
            b = torch.from_numpy(system["b"]).to(DEV)
            x, st, r = s.solve(b)
            assert st == bcs.BCS_OK
            rng = np.random.default_rng(5)
            sys2 = synth.perturb(system, rng, 0.02)
            s.set_values(*(torch.from_numpy(sys2[k]).to(DEV) for k in ("diag", "upper", "lower")))
            z3 = s.precond(vt).cpu().numpy()
            res[graph] = (z1, z2, launches, x.cpu().numpy(), z3)
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert np.array_equal(res[1][0], res[1][1])
    assert res[0][2] == res[1][2]
    assert np.array_equal(res[0][3], res[1][3])
    assert np.array_equal(res[0][4], res[1][4])
    assert not np.array_equal(res[1][0], res[1][4])


SWEEP_COARSE = [
    ("density 16^3", lambda: synth.density(16, seed=0), dict(coarse_dense_max=1)),
    ("pressure 12^3 coarse 200", lambda: synth.pressure(12, seed=1), dict(coarse_dense_max=1, coarse_size=200)),
    ("density 10^3 coarse 200 sweeps 3", lambda: synth.density(10, seed=5),
     dict(coarse_dense_max=1, coarse_size=200, coarse_sweeps=3)),
]


@pytest.mark.parametrize("name,gen,kw", SWEEP_COARSE, ids=[c[0] for c in SWEEP_COARSE])
def test_coarse_smoother_sweeps_fp64_parity(name, gen, kw):
    """The coarsest level solved by block-Jacobi sweeps instead of the dense
    inverse (coarse_kind 1, taken when rows * n exceeds coarse_dense_max):
    the hierarchy is bit-exact with the reference and marks the coarsest
    level for sweeps; the FP64 V-cycle agrees to 1e-12; FP32 storage to the
    FP32 tolerance."""
    system = gen()
    ref = oracle.ldu_to_bsr(system)
    amg = oracle.Amg(ref, oracle_cfg(**kw))
    assert amg.status == 0 and amg.info(amg.levels - 1)["coarse_kind"] == 1
    v = np.random.default_rng(8).standard_normal(system["b"].shape)
    z_ref = amg.vcycle(v)
    with bcs.Solver(system["n"], precision=bcs.BCS_PREC_FP64, **kw) as s:
        s.load(system, device=DEV)
        compare_hierarchy(s, amg, system["n"], 1)
        assert s.level(s.levels - 1)["coarse_kind"] == 1
        z = s.precond(torch.from_numpy(v).to(DEV)).cpu().numpy()
    assert np.abs(z - z_ref).max() <= 1e-12 * np.abs(z_ref).max()
    with bcs.Solver(system["n"], precision=bcs.BCS_PREC_FP32, **kw) as s:
        s.load(system, device=DEV)
        z32 = s.precond(torch.from_numpy(v).to(DEV)).cpu().numpy()
    assert np.linalg.norm(z32 - z_ref) <= 2e-5 * np.linalg.norm(z_ref)
