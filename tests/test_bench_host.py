"""Host-side logic of bench.py and the flow-state generator, without a GPU:
the clock summary (median SM clock, throttle reasons) from nvidia-smi CSV
lines, the reference arm's JSON line (the oracle timed on the host cores),
and the physical validity of synth.flow's states and geometry."""
import json
import os
import subprocess
import sys

import numpy as np

import bench
from paper_2403_07882_b300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` runs the oracle (one step: a full solve of
    the 64^3 sample) and prints exactly one JSON line with the launch
    contract's keys, on the native arm's metric and workload."""
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["config"]["workload"] == bench.WORKLOAD
    assert d["unit"] == "ms" and d["higher_is_better"] is False and d["n_gpus"] == 1
    assert d["steps"] == 1 and d["warmup"] == 0 and d["value"] > 0 and d["vs_baseline"] is None
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_clock_summary_from_csv_lines():
    c = bench.ClockSampler(0)
    c.lines = ["0, 2032, 2032, 850.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 2010, 2032, 910.4, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 1995, 2032, 930.0, 0x4, Not Active, Not Active, Not Active, Active",
               "garbage line", ""]
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2010.0 and s["sm_max_mhz"] == 2032.0
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = ["0, 1500, 2032, 500, 0x40, Not Active, Active, Not Active, Not Active"]
    assert bench.ClockSampler.summary(c)["reasons"] == ["hw_thermal_slowdown"]
    c.lines = []
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_flow_states_and_geometry_are_physical():
    for skew in (False, True):
        fl = synth.flow(7, 5, 4, seed=3, skew=skew)
        Q, g = fl["Q"], fl["gamma"]
        rho = Q[:, 0]
        u = Q[:, 1:4] / rho[:, None]
        p = (g - 1) * (Q[:, 4] - 0.5 * rho * (u * u).sum(1))
        assert np.all(rho > 0) and np.all(p > 0)
        assert np.allclose(np.linalg.norm(fl["normal"], axis=1), 1.0, rtol=1e-14)
        assert np.all(fl["area"] > 0) and np.all(fl["dist"] > 0)
        assert np.all(fl["owner"] < fl["neighbour"])
        assert fl["n_faces"] == 6 * 5 * 4 + 7 * 4 * 4 + 7 * 5 * 3   # internal faces of a 7x5x4 grid
    a, b = synth.flow(5, seed=1), synth.flow(5, seed=1)
    assert all(np.array_equal(a[k], b[k]) for k in ("Q", "normal", "area", "dist", "b"))
