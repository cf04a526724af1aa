"""Launch statistics and CUDA-event timing of the library (cfg.profile):
the per-kernel table, the per-kind totals and the per-level attribution
agree with one another on a full setup + solve."""
import numpy as np
import pytest

from paper_2403_07882_b300 import bcs, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def profiled_step(system, **cfg):
    s = bcs.Solver(system["n"], profile=1, **cfg)
    s.load(system, device=DEV)
    b = torch.from_numpy(system["b"]).to(DEV)
    x, st, res = s.solve(b)
    assert st == bcs.BCS_OK, res
    return s


@pytest.mark.parametrize("cfg", [dict(), dict(pmode=bcs.BCS_P_SMOOTHED), dict(precision=bcs.BCS_PREC_FP64)],
                         ids=["fp32", "fp32-smoothed-P", "fp64"])
def test_level_times_add_up_to_kind_totals(cfg):
    system = synth.density(16, seed=0)
    with profiled_step(system, **cfg) as s:
        kinds = s.stats()["kinds"]
        per_level = s.level_times()
        assert len(per_level) == s.levels >= 3
        # the V-cycle's kernels all belong to a level
        for kind in ("jacobi_sweep", "residual", "transfer", "coarse_solve"):
            n = sum(t[kind]["launches"] for t in per_level if kind in t)
            ms = sum(t[kind]["ms"] for t in per_level if kind in t)
            assert n == kinds[kind]["launches"] > 0, kind
            assert ms == pytest.approx(kinds[kind]["ms"], rel=1e-6), kind
        # the setup's level loop holds most of its work (structure building
        # before it belongs to no level)
        for kind in ("setup_aggregation", "setup_galerkin", "setup_inverse"):
            n = sum(t[kind]["launches"] for t in per_level if kind in t)
            assert 0 < n <= kinds[kind]["launches"], kind
        # every level but the coarsest smooths, restricts and prolongs and
        # is aggregated; the coarsest holds the dense coarse solve
        for l, t in enumerate(per_level[:-1]):
            assert t["jacobi_sweep"]["launches"] > 0 and t["transfer"]["launches"] > 0, l
            assert t["residual"]["launches"] > 0 and t["setup_aggregation"]["ms"] > 0, l
            assert t["jacobi_sweep"]["bytes"] > 0 and t["jacobi_sweep"]["ms"] > 0, l
        assert per_level[-1]["coarse_solve"]["launches"] > 0
        assert "jacobi_sweep" not in per_level[-1]
        # the FP64 outer products, the value gather and the Krylov vector
        # work belong to no level
        for t in per_level:
            assert not any(k in t for k in ("spmv_fp64", "ldu_to_bsr", "blas1"))


def test_level_times_reset_and_range():
    system = synth.density(8, seed=1)
    with profiled_step(system) as s:
        assert s.level_times()[0]
        s.reset_stats()
        assert all(t == {} for t in s.level_times())
        for bad in (-1, 64):
            with pytest.raises(bcs.BcsError) as e:
                bcs.bcs_get_level_times(s.h, bad)
            assert e.value.status == bcs.BCS_EINVAL


def test_no_level_times_without_profiling():
    system = synth.density(8, seed=1)
    with bcs.Solver(5) as s:
        s.load(system, device=DEV)
        x, st, _ = s.solve(torch.from_numpy(system["b"]).to(DEV))
        assert st == bcs.BCS_OK
        assert s.stats()["launches"] > 0
        assert all(t == {} for t in s.level_times())
