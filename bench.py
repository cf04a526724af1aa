"""Benchmark: time-to-1e-8 relative residual of the block-coupled solve.

Workload: density-based coupled system, 5x5 FP64 blocks on a 128^3 hex grid
(2,097,152 cells, 10,485,760 unknowns, 14,581,760 blocks; seed 2). One step
is the whole hot path on one batch: LDU face addressing -> block CSR,
LDU values -> block CSR, full aggregation-AMG setup, and FGMRES(30) with the
FP32-stored AMG preconditioner inside FP64 outer iterations, to a true
relative residual of 1e-8, from x0 = 0. The same step with an all-FP64 AMG is
timed beside it (the mixed-vs-FP64 comparison), and so is the values-only
resetup.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU reference implementation (the oracle)
on the machine's host cores on a bounded sample of the same workload.
Inputs stay larger than L2 (2.9 GB of matrix values), so no L2 flush is
needed between steps.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-8 rel. residual (mixed FP32-AMG in FP64 FGMRES(30)), density-based 128^3 5x5"
WORKLOAD = "density-based coupled system, 5x5 FP64 blocks, 128^3 hex grid (2.1M cells, 10.5M unknowns), seed 2"
SIDE = 128
SAMPLE_SIDE = 64


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--side", type=int, default=SIDE)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-full", action="store_true",
                   help="also run the oracle (OpenMP build, then one core) on the full-size system once "
                        "(minutes, ~20 GB host memory)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp64", action="store_true", help="skip the all-FP64 comparison run")
    p.add_argument("--no-assembly", action="store_true", help="skip the density-based assembly measurement")
    p.add_argument("--workload", default="density128",
                   choices=["density128", "density16", "pressure64", "knn", "serve"],
                   help="density128: the benchmark line; density16 / pressure64: the small density-based and "
                        "the pressure-based systems; knn: unstructured resetup sequence; serve: serving mix")
    p.add_argument("--knn-side", type=int, default=160)
    p.add_argument("--serve-cases", type=int, default=32)
    p.add_argument("--serve-requests", type=int, default=2000)
    p.add_argument("--serve-warmup", type=int, default=200)
    p.add_argument("--serve-rate", type=float, default=200.0)
    p.add_argument("--serve-max-cells", type=float, default=3e6)
    p.add_argument("--serve-slots", type=int, default=8)
    p.add_argument("--serve-oracle", type=int, default=64,
                   help="serving: requests of the smaller cases solved in one mix and checked against the oracle")
    p.add_argument("--serve-oracle-max-cells", type=float, default=2e5,
                   help="serving: largest case the oracle parity subset draws from")
    p.add_argument("--serve-solver", default="fgmres", choices=["fgmres", "bicgstab"],
                   help="serving: Krylov solver of every case")
    p.add_argument("--serve-batch", type=int, default=1,
                   help="serving: solve up to this many resident cases' requests together (1: off)")
    p.add_argument("--serve-budget-gb", type=float, default=0.0,
                   help="HBM budget of the server in GB (0: the default, 80 %% of free memory)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(value, device):
    """Largest per-rank value (the step time of the slowest replica); every
    rank gets it. Needs an initialised process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d["hbm_gbs"], "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


SETUP_KINDS = ("setup_aggregation", "setup_galerkin", "setup_inverse", "scan_sort", "cast")
CYCLE_KINDS = ("jacobi_sweep", "residual", "transfer", "coarse_solve")


def level_table(solver):
    """Per hierarchy level of one profiled step: its size, the CUDA-event
    time of its setup work (aggregation of its rows, the Galerkin product
    forming the next level, its block inverses, sorts and FP32 copies) and
    of its V-cycle kernels with their algorithmic GB/s."""
    out = []
    for l, t in enumerate(solver.level_times()):
        info = solver.level_info(l)
        row = {"level": l, "rows": info["rows"], "nnz": info["nnz"],
               "setup_ms": round(sum(t[k]["ms"] for k in SETUP_KINDS if k in t), 4)}
        for k in CYCLE_KINDS:
            if k in t:
                v = t[k]
                row[k] = {"ms": round(v["ms"], 4), "launches": v["launches"],
                          "GBps": round(v["bytes"] / (v["ms"] * 1e6), 1) if v["ms"] > 0 else None}
        out.append(row)
    return out


def kernel_source_digest(path, func):
    """SHA-256 of the text of the __global__ or __device__ function `func` in
    `path` (from its definition line to the first line that closes it at
    column 0)."""
    import hashlib
    lines = open(path).read().splitlines()
    start = next(i for i, l in enumerate(lines)
                 if ("__global__" in l or "__device__" in l) and (" " + func + "(") in l)
    end = next(i for i in range(start, len(lines)) if lines[i] == "}")
    return hashlib.sha256("\n".join(lines[start:end + 1]).encode()).hexdigest()


def entry_digest(e):
    """Digest of a profiles/traffic.json entry's kernel: its device-function
    body ("function") and, when named, the __global__ wrapper that launches
    it ("wrapper"), concatenated."""
    d = kernel_source_digest(os.path.join(ROOT, e["source"]), e["function"])
    if e.get("wrapper"):
        import hashlib
        d = hashlib.sha256((d + kernel_source_digest(os.path.join(ROOT, e["source"]), e["wrapper"])).encode()).hexdigest()
    return d


def measured_traffic(kernel, bytes_per_launch):
    """DRAM bytes per launch of `kernel`, from the committed ncu summary
    (profiles/traffic.json: DRAM bytes over algorithmic bytes of a captured
    launch), scaled to this run's algorithmic bytes per launch; None when
    absent or when the kernel's source text changed since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            entries = json.load(f)
        e = entries[kernel]
        if entry_digest(e) != e["sha256"]:
            return None
    except (OSError, ValueError, KeyError, StopIteration):
        return None
    return e["dram_over_algorithmic"] * bytes_per_launch


# --------------------------------------------------------------- CPU (oracle)
def host_info():
    """Host CPU model name and the number of usable cores."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"cpu_model": model, "nproc": len(os.sched_getaffinity(0))}


def oracle_run(system, omp=False):
    """One oracle time-to-solution (LDU -> BSR, AMG setup, FGMRES(30) + AMG
    to 1e-8 from x0 = 0): (times in ms, x, result dict). omp selects the
    OpenMP build of the same source (identical results)."""
    import oracle
    oracle.use_openmp(omp)
    try:
        t0 = time.perf_counter()
        ref = oracle.ldu_to_bsr(system)
        amg = oracle.Amg(ref, oracle.config())
        t1 = time.perf_counter()
        x, res, _ = oracle.solve(ref, system["b"], cfg=oracle.config(), amg=amg)
        t2 = time.perf_counter()
    finally:
        oracle.use_openmp(False)
    return {"setup_ms": (t1 - t0) * 1e3, "solve_ms": (t2 - t1) * 1e3, "total_ms": (t2 - t0) * 1e3}, x, res


def oracle_leg(system, cfg_kw, omp=False, spmv_reps=10, resetup=True):
    """The oracle's own times on one system (host cores; omp: the OpenMP
    build of the same source): FP64 SpMV (median of spmv_reps calls), full
    AMG setup, values-only resetup with the same values, and the solve to
    1e-8 from x0 = 0 with the given configuration. Returns (times, x)."""
    import oracle
    oracle.use_openmp(omp)
    try:
        ref = oracle.ldu_to_bsr(system)
        xv = np.random.default_rng(0).uniform(-1, 1, system["b"].shape)
        sp = []
        for _ in range(spmv_reps):
            t0 = time.perf_counter()
            oracle.spmv(ref, xv)
            sp.append((time.perf_counter() - t0) * 1e3)
        cfg = oracle.config(**cfg_kw)
        t0 = time.perf_counter()
        amg = oracle.Amg(ref, cfg)
        t1 = time.perf_counter()
        out = {"spmv_ms": statistics.median(sp), "setup_ms": (t1 - t0) * 1e3}
        if resetup:
            t0 = time.perf_counter()
            amg.resetup(ref["val"])
            out["resetup_ms"] = (time.perf_counter() - t0) * 1e3
        t0 = time.perf_counter()
        x, res, _ = oracle.solve(ref, system["b"], cfg=cfg, amg=amg)
        out["solve_ms"] = (time.perf_counter() - t0) * 1e3
        out.update(status=res["status"], iters=res["iters"],
                   rel_res_true=float(np.linalg.norm(system["b"] - oracle.spmv(ref, x)) / np.linalg.norm(system["b"])))
        return out, x
    finally:
        oracle.use_openmp(False)


def oracle_sample(side=SAMPLE_SIDE):
    """Oracle time-to-solution on the same generator at side^3, in ms."""
    from paper_2403_07882_b300 import synth
    t, _, res = oracle_run(synth.density(side, seed=2))
    return t["total_ms"], res


def gpu_error_arms(system, x_ref, dev):
    """Each GPU arm of the benchmark on `system`, solved to 1e-8 from x0 = 0:
    ||x - x_oracle|| / ||x_oracle|| and the true relative residual recomputed
    with the oracle's FP64 SpMV."""
    import torch
    import oracle
    from paper_2403_07882_b300 import bcs
    ref = oracle.ldu_to_bsr(system)
    arms = {"mixed_fp32_amg": dict(precision=bcs.BCS_PREC_FP32),
            "fp64_amg": dict(precision=bcs.BCS_PREC_FP64),
            "bf16_amg": dict(precision=bcs.BCS_PREC_BF16),
            "dilu_fp32": dict(precision=bcs.BCS_PREC_FP32, smoother=bcs.BCS_SMOOTH_DILU),
            "sgs_fp32_no_amg": dict(precision=bcs.BCS_PREC_FP32, precond=bcs.BCS_PC_SGS, maxiter=5000)}
    bn = np.linalg.norm(system["b"])
    out = {}
    for name, cfg in arms.items():
        with bcs.Solver(system["n"], **cfg) as s:
            s.load(system, device=dev)
            x, st, res = s.solve(torch.from_numpy(system["b"]).to(dev))
            x = x.cpu().numpy()
        out[name] = {"status": st, "iters": res["iters"],
                     "rel_err_x_vs_oracle": float(np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref)),
                     "rel_res_true": float(np.linalg.norm(system["b"] - oracle.spmv(ref, x)) / bn)}
    return out


def cpu_baseline_entry(side, dev=None, full=False):
    """The oracle on the host cores: single-threaded (the baseline value) and
    its OpenMP build on every core, both on the same generator at 64^3,
    their time scaled to side^3 by cell count (a model: the same iteration
    count and a setup linear in the cells); with full=True also measured at
    side^3 itself (minutes). With dev, every GPU arm is solved on the 64^3
    system and compared with the oracle's solution."""
    from paper_2403_07882_b300 import synth
    system = synth.density(SAMPLE_SIDE, seed=2)
    scale = (side / SAMPLE_SIDE) ** 3
    t1, x_ref, res = oracle_run(system)
    tn, x_omp, res_omp = oracle_run(system, omp=True)
    host = host_info()
    entry = {"value": t1["total_ms"] * scale, "unit": "ms", "cores": 1, "kind": "oracle", "modelled": True,
             "sample": f"full oracle solve (LDU->BSR, AMG setup, FGMRES(30)+AMG to 1e-8, {res['iters']} iterations) "
                       f"of the same generator at {SAMPLE_SIDE}^3 = 1/{scale:.0f} of the cells, "
                       f"{t1['total_ms'] / 1e3:.1f} s single-threaded; value = that time x{scale:.0f} by cell count "
                       f"(modelled, not measured at {side}^3)",
             "host": host,
             "measured_sample": dict(side=SAMPLE_SIDE, iters=res["iters"], **t1),
             "oracle_omp": dict(cores=host["nproc"], value=tn["total_ms"] * scale, modelled=True,
                                identical_to_single_thread=bool(np.array_equal(x_ref, x_omp)),
                                parallel_part="row loops of the SpMV and the smoother sweeps, element-wise vector "
                                              "updates; the AMG setup and the dot products stay serial",
                                measured_sample=dict(side=SAMPLE_SIDE, iters=res_omp["iters"], **tn))}
    if full:
        big = synth.density(side, seed=2)
        tf, _, rf = oracle_run(big, omp=True)
        entry["full_size_omp"] = dict(side=side, cores=host["nproc"], iters=rf["iters"],
                                      rel_res_final=rf["rel_res_final"], **tf)
        ts, _, rs = oracle_run(big)
        entry["full_size_single_thread"] = dict(side=side, cores=1, iters=rs["iters"],
                                                rel_res_final=rs["rel_res_final"], **ts)
    if dev is not None:
        entry["gpu_error_vs_oracle"] = {"system": f"density-based {SAMPLE_SIDE}^3, seed 2 (the sample above)",
                                        "arms": gpu_error_arms(system, x_ref, dev)}
    return entry


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    times = []
    res = None
    for i in range(args.warmup + args.steps):
        ms, res = oracle_sample()
        if i >= args.warmup:
            times.append(ms)
    scale = (args.side / SAMPLE_SIDE) ** 3
    value = statistics.mean(times) * scale
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(times),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "solver": "FGMRES(30) + aggregation AMG, FP64 oracle"},
            "cpu_baseline": {"value": value, "unit": "ms", "cores": 1, "kind": "oracle", "modelled": True,
                             "host": host_info(),
                             "sample": f"each step: full oracle solve of the same generator at {SAMPLE_SIDE}^3 "
                                       f"(1/{scale:.0f} of the cells, {res['iters']} iterations), "
                                       f"scaled x{scale:.0f} by cell count (modelled, not measured at full size)"},
            "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ native
def run_native(args):
    import torch
    from paper_2403_07882_b300 import bcs, synth

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    system = synth.density(args.side, seed=2)
    C, F, n = system["n_cells"], system["n_faces"], 5
    keys = ("owner", "neighbour", "diag", "upper", "lower", "b")
    d = {k: torch.from_numpy(system[k]).to(dev) for k in keys}
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def step(s, inp, x, zero_x=True):
        s.set_structure(C, inp["owner"], inp["neighbour"])
        s.set_values(inp["diag"], inp["upper"], inp["lower"])
        if zero_x:
            x.zero_()
        return s.solve(inp["b"], x)

    def timed(s, inp, x, steps, warmup, zero_x=True):
        for _ in range(warmup):
            _, st, res = step(s, inp, x, zero_x)
            assert st == bcs.BCS_OK, res
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.reset_stats()
        results = []
        e0.record(stream)
        for _ in range(steps):
            _, st, res = step(s, inp, x, zero_x)
            assert st == bcs.BCS_OK, res
            results.append(res)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return e0.elapsed_time(e1) / steps, results, s.stats()

    # mixed precision (the headline). One untimed step with CUDA events on
    # every launch gives the per-kernel table and the dominant kernel; inside
    # the timed region only that kernel's kind carries events (so event
    # records do not slow the step, and the cycle can still run as a CUDA
    # graph when the dominant kernel is outside it).
    x = torch.zeros_like(d["b"])
    with bcs.Solver(n, precision=bcs.BCS_PREC_FP32, profile=1) as sp:
        step(sp, d, x)
        torch.cuda.synchronize()
        sp.reset_stats()
        step(sp, d, x)
        ktimes = sp.kernel_times()
        kinds = sp.stats()["kinds"]
        per_level = level_table(sp)
    top_name = max(ktimes.items(), key=lambda kv: kv[1]["ms"])[0]
    live_kinds = 1 << ktimes[top_name]["kind"]
    with ClockSampler(local) as clk:
        with bcs.Solver(n, precision=bcs.BCS_PREC_FP32, profile=1, profile_kinds=live_kinds) as s:
            ms_mixed, res_mixed, stats = timed(s, d, x, args.steps, args.warmup)
            live = s.kernel_times()
            # values-only resetup (Alg. 1: replace coefficients on fixed sparsity)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.set_values(d["diag"], d["upper"], d["lower"])
            e1.record(stream)
            torch.cuda.synchronize()
            resetup_ms = e0.elapsed_time(e1)
    clocks = clk.summary()
    # the same step without any per-kernel events: the V-cycle replays as a
    # CUDA graph and each FGMRES restart cycle runs on the device (events on
    # the dominant kernel's launches, needed for the live roofline above,
    # switch both off)
    with bcs.Solver(n, precision=bcs.BCS_PREC_FP32) as su:
        ms_plain, res_plain, stats_plain = timed(su, d, x, args.steps, args.warmup)
    # all-FP64 comparison (same step, FP64 AMG) and BF16-stored AMG
    ms_fp64, res_fp64, ms_bf16, res_bf16, ms_dilu, res_dilu = None, None, None, None, None, None
    ms_sgs, res_sgs = None, None
    if not args.no_fp64:
        with bcs.Solver(n, precision=bcs.BCS_PREC_FP64) as s64:
            ms_fp64, res_fp64, _ = timed(s64, d, x, max(1, min(args.steps, 3)), 1)
        with bcs.Solver(n, precision=bcs.BCS_PREC_BF16) as s16:
            ms_bf16, res_bf16, _ = timed(s16, d, x, max(1, min(args.steps, 3)), 1)
        with bcs.Solver(n, precision=bcs.BCS_PREC_FP32, smoother=bcs.BCS_SMOOTH_DILU) as sd:
            ms_dilu, res_dilu, _ = timed(sd, d, x, max(1, min(args.steps, 3)), 1)
        with bcs.Solver(n, precision=bcs.BCS_PREC_FP32, precond=bcs.BCS_PC_SGS, maxiter=5000) as ss:
            ms_sgs, res_sgs, _ = timed(ss, d, x, max(1, min(args.steps, 3)), 1)

    # end to end through the C ABI with pinned host buffers; the zero
    # initial guess is the solver's (x0_zero), so x is only written back
    e2e = None
    if not args.no_e2e:
        h = {k: torch.from_numpy(system[k]).pin_memory() for k in keys}
        xh = torch.empty_like(h["b"]).pin_memory()
        h2d = sum(h[k].numel() * h[k].element_size() for k in keys)
        with bcs.Solver(n, precision=bcs.BCS_PREC_FP32, x0_zero=1) as se:
            ms_e2e, _, _ = timed(se, h, xh, max(1, min(args.steps, 3)), 1, zero_x=False)
        e2e = {"value": ms_e2e, "unit": "ms", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(xh.numel() * 8)}

    assembly = None if args.no_assembly else assembly_entry(args.side, dev, args.steps)
    packing = None if args.no_assembly else packing_entry(system, dev, args.steps)

    ms_max = max_over_ranks(ms_mixed, dev) if world > 1 else ms_mixed
    if rank != 0:
        return

    peak, peak_kind = peaks()
    # the dominant kernel's events inside the timed region
    top = live[top_name]
    per_launch_bytes = top["bytes"] / max(top["launches"], 1)
    per_launch_ms = top["ms"] / max(top["launches"], 1)
    achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
    traffic = measured_traffic(top_name, per_launch_bytes)
    roofline = {"bound": "hbm", "kernel": top_name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind + " (copy bandwidth)",
                "frac_of_nominal_7700": achieved / 7700.0,
                "launches_in_timed_region": top["launches"], "bytes_per_launch": per_launch_bytes,
                "ms_per_launch": per_launch_ms}
    # per-kind and per-kernel tables: one profiled step outside the timed region
    breakdown = {k: {"ms_per_step": v["ms"], "launches_per_step": v["launches"],
                     "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None}
                 for k, v in kinds.items() if v["launches"]}
    line = {
        "metric": METRIC, "value": ms_max, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 outer / f32 AMG", "data": "synthetic",
        "config": {"workload": WORKLOAD, "solver": "FGMRES(30) + aggregation AMG (2 matching passes, "
                                                   "tentative P, block-Jacobi 2+2 sweeps, w=0.8)",
                   "precision": "FP32-stored AMG, FP64 outer SpMV / Gram-Schmidt / Hessenberg",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (2.9 GB of FP64 block values); no flush needed",
                   "step": "set_structure + set_values (full AMG setup) + solve, device-resident inputs"},
        "host_syncs_per_solve": {"timed (host-driven loop, events on)": res_mixed[-1]["host_syncs"],
                                 "uninstrumented (device loops)": res_plain[-1]["host_syncs"],
                                 "iters": res_plain[-1]["iters"]},
        "uninstrumented": {"value": ms_plain, "unit": "ms", "iters": res_plain[-1]["iters"],
                           "gpu_launches_per_step": stats_plain["launches"] / args.steps,
                           "note": "the same step with no per-kernel events: graph-replayed V-cycle and "
                                   "device-resident FGMRES restart cycles"},
        "iters": res_mixed[-1]["iters"], "rel_res_final": res_mixed[-1]["rel_res_final"],
        "levels": res_mixed[-1]["levels"],
        "fp64": None if ms_fp64 is None else {"value": ms_fp64, "unit": "ms", "iters": res_fp64[-1]["iters"],
                                              "speedup_mixed_vs_fp64": ms_fp64 / ms_mixed},
        "bf16": None if ms_bf16 is None else {"value": ms_bf16, "unit": "ms", "iters": res_bf16[-1]["iters"],
                                              "rel_res_final": res_bf16[-1]["rel_res_final"]},
        "dilu": None if ms_dilu is None else {"value": ms_dilu, "unit": "ms", "iters": res_dilu[-1]["iters"],
                                              "rel_res_final": res_dilu[-1]["rel_res_final"],
                                              "smoother": "multicolour block DILU, FP32 storage"},
        "sgs": None if ms_sgs is None else {"value": ms_sgs, "unit": "ms", "iters": res_sgs[-1]["iters"],
                                            "rel_res_final": res_sgs[-1]["rel_res_final"],
                                            "preconditioner": "GMRES + multicolour block SGS (LU-SGS form), "
                                                              "FP32 storage, no AMG"},
        "resetup_ms": resetup_ms,
        "roofline": roofline,
        "kernel_breakdown": breakdown,
        "per_level": per_level,
        "kernels": {k: {"ms_per_step": round(v["ms"], 4), "launches_per_step": v["launches"],
                        "GBps": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1) if v["ms"] > 0 else None}
                    for k, v in sorted(ktimes.items(), key=lambda kv: -kv[1]["ms"])[:40]},
        "gpu_launches": int(stats["launches"]),
        "gpu_launches_per_step": stats["launches"] / args.steps,
        "clocks": clocks,
        "e2e": e2e,
        "assembly": assembly,
        "packing": packing,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_entry(args.side, dev=dev, full=args.cpu_full)
    print(json.dumps(line), flush=True)


# FP64 thread instructions (DADD + DMUL + DFMA) of the assembly, measured by
# ncu on the 64^3 mesh (profiles/assembly_density64.md): k_cell_prims and
# k_assemble_cells 481 per cell (a cell with its face sides), k_face_lambda
# 42 per face. Peak: 296 DFMA thread instructions per cycle on the GPU (ncu's
# sustained peak of sm__sass_thread_inst_executed_op_dfma_pred_on) at the
# 2032 MHz maximum SM clock.
ASSEMBLY_FP64_OPS = {"per_cell": 481.0, "per_face": 42.0}
FP64_PEAK_OPS = 296 * 2032e6


def assembly_entry(side, dev, reps):
    """Density-based assembly (Sec. 2.1) on the side^3 mesh: the assembly
    kernels alone (LDU blocks on the device) and one nonlinear iteration
    (assembly straight into the solver's values, values-only resetup, solve)."""
    import torch
    from paper_2403_07882_b300 import bcs, synth
    fl = synth.flow(side, seed=5)
    C, F = fl["n_cells"], fl["n_faces"]
    g = {k: torch.from_numpy(np.ascontiguousarray(fl[k])).to(dev)
         for k in ("owner", "neighbour", "Q", "area", "normal", "dist", "b")}
    stream = torch.cuda.current_stream()
    reps = max(3, reps)
    with bcs.Solver(5, profile=1, profile_kinds=bcs.kind_mask("assembly")) as s:
        s.set_structure(C, g["owner"], g["neighbour"])
        out = (torch.empty((C, 5, 5), dtype=torch.float64, device=dev),
               torch.empty((F, 5, 5), dtype=torch.float64, device=dev),
               torch.empty((F, 5, 5), dtype=torch.float64, device=dev))
        prm = bcs.bcs_flow_params_default()
        for _ in range(2):
            bcs.bcs_assemble_density(s.h, g["Q"], g["area"], g["normal"], g["dist"], prm, *out)
        torch.cuda.synchronize()
        s.reset_stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            bcs.bcs_assemble_density(s.h, g["Q"], g["area"], g["normal"], g["dist"], prm, *out)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        kt = s.kernel_times()
        # one nonlinear iteration: assemble into the solver's values (the first
        # call runs the full setup), then values-only resetup + solve
        s.assemble_density(g["Q"], g["area"], g["normal"], g["dist"], to_values=True)
        x = torch.zeros_like(g["b"])
        torch.cuda.synchronize()
        e0.record(stream)
        iters = []
        for _ in range(reps):
            s.assemble_density(g["Q"], g["area"], g["normal"], g["dist"], to_values=True)
            x.zero_()
            _, st, res = s.solve(g["b"], x)
            assert st == bcs.BCS_OK, res
            iters.append(res["iters"])
        e1.record(stream)
        torch.cuda.synchronize()
        ms_nl = e0.elapsed_time(e1) / reps
    kernels = {}
    for name, v in kt.items():
        if not v["launches"]:
            continue
        per = v["ms"] / v["launches"]
        kernels[name] = {"ms_per_launch": per, "GBps": v["bytes"] / v["launches"] / (per * 1e-3) / 1e9}
    fp64_ops = ASSEMBLY_FP64_OPS["per_cell"] * C + ASSEMBLY_FP64_OPS["per_face"] * F
    peak_ops = FP64_PEAK_OPS
    return {"workload": f"density-based assembly (Sec. 2.1, Eqs. approxJac1/2), {side}^3 hex mesh, "
                        f"{C} cells, {F} faces, LDU blocks on the device",
            "ms": ms, "kernels": kernels,
            "roofline": {"bound": "alu", "unit": "FP64 thread instructions/s", "achieved": fp64_ops / (ms * 1e-3),
                         "peak": peak_ops, "frac": fp64_ops / (ms * 1e-3) / peak_ops,
                         "peak_source": "296 DFMA thread instructions per cycle (ncu sustained peak) x 2032 MHz",
                         "ops_per_assembly": fp64_ops,
                         "ops_source": "DADD + DMUL + DFMA thread instructions counted by ncu on 64^3, "
                                       "481 per cell + 42 per face"},
            "nonlinear_iteration_ms": ms_nl, "nonlinear_iteration":
                "assembly into the solver's values + values-only resetup + FGMRES solve to 1e-8",
            "iters": iters[-1]}


def packing_entry(system, dev, reps):
    """Coefficients from segregated field couplings to block AoS (Alg. 1 step
    5) on the benchmark system: density-based, fields (rho, rhoU, rhoE), nine
    couplings, all on the device. LDU blocks out (HBM-bound copy: every value
    read once and written once), and straight into the solver's block-CSR
    values (step 5 fused with the LDU -> block-CSR permutation)."""
    import torch
    from paper_2403_07882_b300 import bcs
    C, F = system["n_cells"], system["n_faces"]
    ncomp = [1, 3, 1]
    off = [0, 1, 4, 5]
    cp = [[tuple(torch.from_numpy(np.ascontiguousarray(system[k][:, off[a]:off[a + 1], off[b]:off[b + 1]])).to(dev)
                 for k in ("diag", "upper", "lower")) for b in range(3)] for a in range(3)]
    stream = torch.cuda.current_stream()
    reps = max(3, reps)
    out = {}
    with bcs.Solver(5, profile=1, profile_kinds=bcs.kind_mask("ldu_to_bsr")) as s:
        s.set_structure(C, torch.from_numpy(system["owner"]).to(dev), torch.from_numpy(system["neighbour"]).to(dev))
        ldu = (torch.empty((C, 5, 5), dtype=torch.float64, device=dev),
               torch.empty((F, 5, 5), dtype=torch.float64, device=dev),
               torch.empty((F, 5, 5), dtype=torch.float64, device=dev))
        for mode in ("ldu", "values"):
            for _ in range(2):
                if mode == "ldu":
                    bcs.bcs_pack_coefficients(s.h, ncomp, cp, *ldu)
            torch.cuda.synchronize()
            s.reset_stats()
            for _ in range(reps):
                if mode == "ldu":
                    bcs.bcs_pack_coefficients(s.h, ncomp, cp, *ldu)
                else:
                    # the first call runs the full setup; the kernel is timed by its events
                    s.pack_coefficients(cp, ncomp, to_values=True)
            torch.cuda.synchronize()
            kt = {k: v for k, v in s.kernel_times().items() if "pack_coefficients" in k}
            (name, v), = kt.items()
            per = v["ms"] / v["launches"]
            bpl = v["bytes"] / v["launches"]
            out[mode] = {"kernel": name, "ms_per_launch": per, "GBps": bpl / (per * 1e-3) / 1e9,
                         "bytes_per_launch": bpl}
    peak, peak_kind = peaks()
    best = out["ldu"]
    return {"workload": f"segregated fields (rho, rhoU, rhoE) -> block AoS coefficients, {C} cells, {F} faces, "
                        f"9 couplings, device-resident",
            "ldu": out["ldu"], "into_values": out["values"],
            "roofline": {"bound": "hbm", "kernel": best["kernel"], "achieved": best["GBps"], "peak": peak,
                         "unit": "GB/s", "frac": best["GBps"] / peak, "peak_source": peak_kind + " (copy bandwidth)"}}


def run_system(args):
    """The 16^3 density-based system (L2-resident: launch-bound, no HBM
    fraction) or the 64^3 pressure-based system with permuted numbering:
    full setup, resetup and solve times per solver and precision, launches
    per solve, median over the timed repetitions."""
    import torch
    from paper_2403_07882_b300 import bcs, synth
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    # (label, solver, AMG precision, reorder, extra options, preconditioner label)
    jac, dilu, sgs = dict(), dict(smoother=bcs.BCS_SMOOTH_DILU), dict(precond=bcs.BCS_PC_SGS, maxiter=5000)
    if args.workload == "density16":
        system, n = synth.density(16, seed=0), 5
        name = "density-based 16^3 5x5 (4,096 cells), seed 0"
        runs = [("fgmres", bcs.BCS_FGMRES, bcs.BCS_PREC_FP32, 0, jac), ("fgmres", bcs.BCS_FGMRES, bcs.BCS_PREC_FP64, 0, jac),
                ("fgmres", bcs.BCS_FGMRES, bcs.BCS_PREC_FP32, 0, dilu),
                ("fgmres", bcs.BCS_FGMRES, bcs.BCS_PREC_FP32, 0, sgs)]
    else:
        system, n = synth.pressure(64, seed=1), 4
        name = "pressure-based 64^3 4x4 (262,144 cells), permuted numbering, seed 1"
        # with and without the internal reverse Cuthill-McKee renumbering
        runs = [("bicgstab", bcs.BCS_BICGSTAB, bcs.BCS_PREC_FP32, 0, jac),
                ("fgmres", bcs.BCS_FGMRES, bcs.BCS_PREC_FP32, 0, jac),
                ("bicgstab", bcs.BCS_BICGSTAB, bcs.BCS_PREC_FP64, 0, jac),
                ("bicgstab", bcs.BCS_BICGSTAB, bcs.BCS_PREC_FP32, 1, jac),
                ("fgmres", bcs.BCS_FGMRES, bcs.BCS_PREC_FP32, 1, jac),
                ("bicgstab", bcs.BCS_BICGSTAB, bcs.BCS_PREC_FP32, 0, dilu),
                ("fgmres", bcs.BCS_FGMRES, bcs.BCS_PREC_FP32, 0, dilu),
                ("fgmres", bcs.BCS_FGMRES, bcs.BCS_PREC_FP32, 0, sgs)]
    keys = ("owner", "neighbour", "diag", "upper", "lower", "b")
    d = {k: torch.from_numpy(system[k]).to(dev) for k in keys}
    ev = lambda: torch.cuda.Event(enable_timing=True)
    pnames = {bcs.BCS_PREC_FP32: "fp32", bcs.BCS_PREC_FP64: "fp64", bcs.BCS_PREC_BF16: "bf16"}
    out = []
    C, F = system["n_cells"], system["n_faces"]
    spmv_bytes = 8.0 * n * n * (C + 2 * F) + 4.0 * (C + 2 * F) + 4.0 * (C + 1) + 16.0 * n * C
    xs = []
    for label, solver, prec, reorder, extra in runs:
        setup, resetup, solve, total, iters, launches, spmv_ms = [], [], [], [], [], [], []
        for rep in range(args.warmup + args.steps):
            with bcs.Solver(n, solver=solver, precision=prec, reorder=reorder, **extra) as s:
                x = torch.zeros_like(d["b"])
                torch.cuda.synchronize()
                e = [ev() for _ in range(5)]
                e[0].record()
                s.set_structure(system["n_cells"], d["owner"], d["neighbour"])
                s.set_values(d["diag"], d["upper"], d["lower"])
                e[1].record()
                s.reset_stats()
                _, st, res = s.solve(d["b"], x)
                e[2].record()
                nl = s.stats()["launches"]
                s.set_values(d["diag"], d["upper"], d["lower"])
                e[3].record()
                y = torch.empty_like(x)
                for _ in range(10):
                    s.spmv(x, y)
                e[4].record()
                torch.cuda.synchronize()
                assert st == bcs.BCS_OK, res
                if rep == args.warmup + args.steps - 1:
                    xs.append(x.cpu().numpy())
                if rep >= args.warmup:
                    setup.append(e[0].elapsed_time(e[1]))
                    solve.append(e[1].elapsed_time(e[2]))
                    total.append(e[0].elapsed_time(e[2]))
                    resetup.append(e[2].elapsed_time(e[3]))
                    iters.append(res["iters"])
                    launches.append(nl)
                    spmv_ms.append(e[3].elapsed_time(e[4]) / 10)
        pc = ("multicolour block SGS (no AMG)" if extra.get("precond") == bcs.BCS_PC_SGS else
              "AMG, multicolour block DILU smoother" if extra.get("smoother") == bcs.BCS_SMOOTH_DILU else
              "AMG, block-Jacobi smoother")
        out.append({"solver": label, "preconditioner": pc, "amg_precision": pnames[prec], "rcm_reorder": bool(reorder),
                    "spmv_fp64_ms": statistics.median(spmv_ms),
                    "spmv_fp64_GBps": spmv_bytes / (statistics.median(spmv_ms) * 1e-3) / 1e9,
                    "time_to_1e-8_ms": statistics.median(total), "setup_ms": statistics.median(setup),
                    "solve_ms": statistics.median(solve), "resetup_ms": statistics.median(resetup),
                    "iters": iters[-1], "launches_per_solve": launches[-1]})
    line = {"impl": "native", "mode": args.workload, "workload": name,
            "step": "structure + values + full setup + solve to 1e-8 from x0 = 0", "runs": out}
    if not args.no_cpu_baseline:
        # the oracle on the host cores with the first arm's solver (FP64
        # throughout): SpMV, full setup, resetup, solve; single-threaded and
        # the OpenMP build; every GPU arm's solution against the oracle's
        okw = dict(solver=runs[0][1])
        t1, x_ref = oracle_leg(system, okw)
        tn, x_omp = oracle_leg(system, okw, omp=True)
        import oracle
        ref = oracle.ldu_to_bsr(system)
        bn = np.linalg.norm(system["b"])
        errs = {}
        for (label, solver, prec, reorder, extra), o, xg in zip(runs, out, xs):
            key = f"{label} / {o['preconditioner']} / {o['amg_precision']}" + (" / rcm" if reorder else "")
            errs[key] = {"rel_err_x_vs_oracle": float(np.linalg.norm(xg - x_ref) / np.linalg.norm(x_ref)),
                         "rel_res_true": float(np.linalg.norm(system["b"] - oracle.spmv(ref, xg)) / bn)}
        line["cpu_baseline"] = {"kind": "oracle", "unit": "ms", "cores": 1, "host": host_info(),
                                "value": t1["setup_ms"] + t1["solve_ms"], "solver": runs[0][0],
                                "sample": "the full system (no sampling): FP64 SpMV (median of 10), AMG setup, "
                                          "values-only resetup, solve to 1e-8",
                                "single_thread": t1,
                                "oracle_omp": dict(cores=host_info()["nproc"], **tn,
                                                   identical_to_single_thread=bool(np.array_equal(x_ref, x_omp))),
                                "gpu_error_vs_oracle": errs}
    print(json.dumps(line), flush=True)


def run_knn(args):
    """Config 4: unstructured k-NN mesh, one full setup, then ten values-only
    resetups (2 % perturbation each, compounding) each followed by a solve."""
    import torch
    from paper_2403_07882_b300 import bcs, synth
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    t0 = time.perf_counter()
    system = synth.knn(args.knn_side, seed=3)
    gen_s = time.perf_counter() - t0
    keys = ("owner", "neighbour", "diag", "upper", "lower", "b")
    d = {k: torch.from_numpy(system[k]).to(dev) for k in keys}
    rng = np.random.default_rng(30)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    out = {"workload": f"knn {args.knn_side}^3 jittered points, k~U{{4..12}}, 5x5 blocks, seed 3",
           "cells": system["n_cells"], "faces": system["n_faces"], "generation_s": gen_s}
    with bcs.Solver(5, precision=bcs.BCS_PREC_FP32) as s:
        s.set_structure(system["n_cells"], d["owner"], d["neighbour"])
        a, b_ = ev(), ev()
        a.record(); s.set_values(d["diag"], d["upper"], d["lower"]); b_.record(); torch.cuda.synchronize()
        out["full_setup_ms"] = a.elapsed_time(b_)
        x = torch.zeros_like(d["b"])
        _, st, res = s.solve(d["b"], x)
        out["first_solve"] = {"status": st, "iters": res["iters"], "ms": res["solve_ms"], "levels": res["levels"]}
        rs, ss, its = [], [], []
        for it in range(10):
            system = synth.perturb(system, rng, 0.02)
            vals = [torch.from_numpy(system[k]).to(dev) for k in ("diag", "upper", "lower")]
            torch.cuda.synchronize()
            a, b_ = ev(), ev()
            a.record(); s.set_values(*vals); b_.record(); torch.cuda.synchronize()
            rs.append(a.elapsed_time(b_))
            x.zero_()
            a, b_ = ev(), ev()
            a.record(); _, st, res = s.solve(d["b"], x); b_.record(); torch.cuda.synchronize()
            assert st == bcs.BCS_OK, res
            ss.append(a.elapsed_time(b_))
            its.append(res["iters"])
        out.update({"resetup_ms_mean": statistics.mean(rs), "solve_ms_mean": statistics.mean(ss),
                    "iters": its, "resetup_over_full_setup": statistics.mean(rs) / out["full_setup_ms"]})
    # the smoother / preconditioner comparison on the last system: full setup
    # and solve to 1e-8 with block Jacobi, DILU and the SGS preconditioner
    vals = [torch.from_numpy(system[k]).to(dev) for k in ("diag", "upper", "lower")]
    cmp_ = {}
    for label, extra in (("block_jacobi_amg", {}), ("dilu_amg", dict(smoother=bcs.BCS_SMOOTH_DILU)),
                         ("sgs_no_amg", dict(precond=bcs.BCS_PC_SGS, maxiter=5000))):
        times = []
        for rep in range(2):
            with bcs.Solver(5, precision=bcs.BCS_PREC_FP32, **extra) as s2:
                s2.set_structure(system["n_cells"], d["owner"], d["neighbour"])
                x2 = torch.zeros_like(d["b"])
                torch.cuda.synchronize()
                a, b_, c_ = ev(), ev(), ev()
                a.record(); s2.set_values(*vals); b_.record(); _, st, res = s2.solve(d["b"], x2); c_.record()
                torch.cuda.synchronize()
                assert st == bcs.BCS_OK, res
                times.append((a.elapsed_time(b_), b_.elapsed_time(c_), res["iters"]))
        setup_ms, solve_ms, it = times[-1]
        cmp_[label] = {"setup_ms": setup_ms, "solve_ms": solve_ms, "time_to_1e-8_ms": setup_ms + solve_ms,
                       "iters": it}
    out["smoother_comparison"] = cmp_
    if not args.no_cpu_baseline:
        # the oracle on the last system: single-threaded SpMV (median of 3),
        # then SpMV, full setup, one values-only resetup and the solve with
        # the OpenMP build (about a minute, some 30 GB of host memory)
        import oracle
        ref = oracle.ldu_to_bsr(system)
        xv = np.random.default_rng(0).uniform(-1, 1, system["b"].shape)
        sp = []
        for _ in range(3):
            t0 = time.perf_counter()
            oracle.spmv(ref, xv)
            sp.append((time.perf_counter() - t0) * 1e3)
        del ref
        tn, x_or = oracle_leg(system, {}, omp=True, spmv_reps=3)
        with bcs.Solver(5, precision=bcs.BCS_PREC_FP32) as s3:
            s3.set_structure(system["n_cells"], d["owner"], d["neighbour"])
            s3.set_values(*vals)
            x3 = torch.zeros_like(d["b"])
            _, st, res = s3.solve(d["b"], x3)
            x3 = x3.cpu().numpy()
        out["cpu_baseline"] = {"kind": "oracle", "unit": "ms", "host": host_info(),
                               "sample": "the last system of the sequence (no sampling)",
                               "single_thread": {"cores": 1, "spmv_ms": statistics.median(sp)},
                               "oracle_omp": dict(cores=host_info()["nproc"], **tn),
                               "gpu_error_vs_oracle": {
                                   "rel_err_x_vs_oracle": float(np.linalg.norm(x3 - x_or) / np.linalg.norm(x_or)),
                                   "gpu_iters": res["iters"]}}
    print(json.dumps({"impl": "native", "mode": "knn", **out}), flush=True)


def host_available_bytes():
    """MemAvailable from /proc/meminfo (physical pages when absent)."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")


def run_serve(args):
    """Config 5: many cases of different sizes, Poisson arrivals, values-only
    resetup + solve per request, admission by HBM budget; p50 / p99 latency.

    Each case's two value sets (the registered one and a 2 % perturbation,
    alternated between its requests) are staged in device memory before the
    clock starts, as the matrices a GPU-side assembly would leave there; the
    per-request work is the values-only resetup and the solve. Two arrival
    processes are run: the configured Poisson rate, and a closed loop that
    keeps every slot busy (the service capacity); when the configured rate is
    above capacity, a third Poisson run at 80 % of capacity gives latencies
    that are not queue growth."""
    import torch
    from paper_2403_07882_b300 import bcs, synth
    torch.cuda.set_device(0)
    ncases = args.serve_cases
    max_cells = args.serve_max_cells
    cells = np.round(np.exp(np.random.default_rng(4).uniform(np.log(5e4), np.log(max_cells), ncases)))
    rng_case = np.random.default_rng(4)
    _ = rng_case.uniform(np.log(5e4), np.log(max_cells), ncases)
    keys = ("diag", "upper", "lower", "b")
    t0 = time.perf_counter()
    budget = int(args.serve_budget_gb * 1e9)
    solver = bcs.BCS_BICGSTAB if args.serve_solver == "bicgstab" else bcs.BCS_FGMRES
    with bcs.Server(budget_bytes=budget, slots=args.serve_slots, batch=args.serve_batch, solver=solver) as srv:
        cases, ids, kinds, small = [], [], [], {}
        for c in range(ncases):
            nx = int(round(cells[c] ** (1.0 / 3.0)))
            nz = max(1, int(round(cells[c] / (nx * nx))))
            if rng_case.uniform() < 0.5:
                sys0, kind = synth.pressure(nx, nx, nz, seed=1000 + c), 4
            else:
                sys0, kind = synth.density(nx, nx, nz, seed=1000 + c), 5
            sys1 = synth.perturb(sys0, rng_case, 0.02)
            ids.append(srv.register(sys0))
            cases.append(tuple({k: torch.from_numpy(v[k]).cuda() for k in keys} for v in (sys0, sys1)))
            kinds.append(kind)
            if sys0["n_cells"] <= args.serve_oracle_max_cells:
                small[c] = (sys0, sys1)  # host copies for the oracle parity subset
            del sys0, sys1
        torch.cuda.synchronize()
        gen_s = time.perf_counter() - t0

        def run(rate, total, warmup, seed, closed=False):
            arr = np.random.default_rng(seed)
            picks = arr.integers(0, ncases, total)
            gaps = arr.exponential(1.0 / rate, total) if rate else np.zeros(total)
            pending, lat, iters = [], [], []
            srv.reset_stats()
            t_next = time.perf_counter()
            measure_from = None
            done_measured = 0
            for r in range(total):
                if closed:
                    # keep at most 2 requests per slot in flight
                    while len(pending) >= 2 * args.serve_slots:
                        rr, t = pending.pop(0)
                        st, res, l, _ = srv.wait(t)
                        assert st in (bcs.BCS_OK, bcs.BCS_REJECTED), (res, srv.last_error())
                        if rr >= warmup and st == bcs.BCS_OK:
                            lat.append(l)
                            iters.append(res["iters"])
                else:
                    t_next += gaps[r]
                    now = time.perf_counter()
                    if t_next > now:
                        time.sleep(t_next - now)
                if r == warmup:
                    measure_from = time.perf_counter()
                c = int(picks[r])
                pending.append((r, srv.submit(ids[c], cases[c][r % 2])))
                if not closed:
                    keep = []
                    for rr, t in pending:
                        st, res, l, _ = srv.wait(t, timeout_ms=0)
                        if st == bcs.BCS_TIMEOUT:
                            keep.append((rr, t))
                        else:
                            assert st in (bcs.BCS_OK, bcs.BCS_REJECTED), (res, srv.last_error())
                            if rr >= warmup and st == bcs.BCS_OK:
                                lat.append(l)
                                iters.append(res["iters"])
                    pending = keep
            for rr, t in pending:
                st, res, l, _ = srv.wait(t)
                assert st in (bcs.BCS_OK, bcs.BCS_REJECTED), (res, srv.last_error())
                if rr >= warmup and st == bcs.BCS_OK:
                    lat.append(l)
                    iters.append(res["iters"])
            elapsed = time.perf_counter() - measure_from
            stats = srv.stats()
            lat = np.array(lat)
            return {"offered_per_s": rate if not closed else None, "requests": total - warmup,
                    "solves_per_s": len(lat) / elapsed,
                    "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                    "mean_ms": float(lat.mean()), "iters_max": int(max(iters)),
                    "evictions": stats["evictions"], "rejected": stats["rejected"],
                    "resident_bytes": stats["resident_bytes"], "budget_bytes": stats["budget_bytes"],
                    "batches": stats["batches"], "batched_requests": stats["batched_requests"],
                    "gpu_timeline": {"window_ms": stats["window_ms"], "busy_frac": stats["busy_frac"],
                                     "overlap2_frac": stats["overlap_frac"],
                                     "mean_requests_in_flight": stats["mean_in_flight"],
                                     "how": "per request: CUDA events on its case's stream before the "
                                            "resetup and after the solve"}}

        n_req, n_warm = args.serve_requests, args.serve_warmup
        configured = run(args.serve_rate, n_warm + n_req, n_warm, 5)
        capacity = run(0.0, n_warm + n_req, n_warm, 6, closed=True)
        below = None
        if args.serve_rate > 0.8 * capacity["solves_per_s"]:
            below = run(0.8 * capacity["solves_per_s"], n_warm + n_req, n_warm, 7)
        parity = None
        if args.serve_oracle > 0 and small and not args.no_cpu_baseline:
            parity = serve_oracle_parity(args, srv, ids, cases, small, solver)
    print(json.dumps({"impl": "native", "mode": "serve", "cases": ncases,
                      "cells_range": [5e4, max_cells], "cells_mean": float(cells.mean()),
                      "block_sizes": {"5": kinds.count(5), "4": kinds.count(4)}, "slots": args.serve_slots,
                      "batch": args.serve_batch, "solver": args.serve_solver,
                      "budget": "default (80 % of free memory)" if budget == 0 else f"{args.serve_budget_gb:g} GB",
                      "inputs": "two value sets per case resident in device memory, alternated per request",
                      "setup_s": gen_s, "configured_rate": configured, "closed_loop_capacity": capacity,
                      "at_80pct_capacity": below, "oracle_parity": parity}), flush=True)


def serve_oracle_parity(args, srv, ids, cases, small, solver):
    """Requests of the smaller cases submitted together (in one mix on all
    slots), each solution checked by the oracle on the host: its true
    relative residual recomputed with the FP64 SpMV, and its distance to the
    oracle's own solution of the same system. Repeats of one (case, value
    set) must return identical solutions."""
    import oracle
    from paper_2403_07882_b300 import bcs
    rng = np.random.default_rng(8)
    keys = sorted(small)
    picks = [(int(keys[rng.integers(0, len(keys))]), int(rng.integers(0, 2))) for _ in range(args.serve_oracle)]
    tickets = [srv.submit(ids[c], cases[c][v]) for c, v in picks]
    got = {}
    identical = True
    for (c, v), t in zip(picks, tickets):
        st, res, _, x = srv.wait(t)
        assert st == bcs.BCS_OK, res
        x = x.cpu().numpy()
        if (c, v) in got:
            identical &= bool(np.array_equal(got[(c, v)], x))
        else:
            got[(c, v)] = x
    okw = dict(solver=solver)
    worst_res, worst_err = 0.0, 0.0
    t0 = time.perf_counter()
    oracle.use_openmp(True)
    try:
        for (c, v), x in got.items():
            sysv = small[c][v]
            ref = oracle.ldu_to_bsr(sysv)
            xo, ores, _ = oracle.solve(ref, sysv["b"], cfg=oracle.config(**okw))
            assert ores["status"] == 0, ores
            bn = np.linalg.norm(sysv["b"])
            worst_res = max(worst_res, float(np.linalg.norm(sysv["b"] - oracle.spmv(ref, x)) / bn))
            worst_err = max(worst_err, float(np.linalg.norm(x - xo) / np.linalg.norm(xo)))
    finally:
        oracle.use_openmp(False)
    return {"requests": len(picks), "distinct_systems": len(got), "cases": len(small),
            "max_cells": args.serve_oracle_max_cells, "repeats_identical": identical,
            "max_rel_res_true_by_oracle": worst_res, "max_rel_err_x_vs_oracle": worst_err,
            "oracle_s": time.perf_counter() - t0, "oracle_cores": host_info()["nproc"]}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "knn":
        run_knn(args)
    elif args.workload in ("density16", "pressure64"):
        run_system(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
