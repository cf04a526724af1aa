"""Serving (continuous batching across cases): every result is bit-identical
whether its case runs alone or interleaved with other cases on several
slots; admission by memory budget evicts idle cases and rejects cases that
can never fit; every solve reaches the 1e-8 true residual."""
import numpy as np
import pytest

import oracle
from paper_2403_07882_b300 import bcs, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def cases():
    return [synth.density(10, seed=1), synth.pressure(8, seed=2), synth.density(12, 9, 7, seed=3),
            synth.random_graph(500, 1500, 3, seed=4)]


def sequences(systems, k=3):
    out = []
    for c, sys0 in enumerate(systems):
        rng = np.random.default_rng(100 + c)
        seq, cur = [], sys0
        for _ in range(k):
            cur = synth.perturb(cur, rng, 0.02)
            seq.append(cur)
        out.append(seq)
    return out


def true_rel(system, x):
    ref = oracle.ldu_to_bsr(system)
    r = system["b"] - oracle.spmv(ref, x)
    return np.linalg.norm(r) / np.linalg.norm(system["b"])


def test_results_identical_alone_and_in_mix():
    systems = cases()
    seqs = sequences(systems)
    alone = []
    for c, system in enumerate(systems):
        with bcs.Server(slots=1) as srv:
            cid = srv.register(system)
            tickets = [srv.submit(cid, s) for s in seqs[c]]
            xs = []
            for t in tickets:
                st, res, lat, x = srv.wait(t)
                assert st == bcs.BCS_OK, res
                xs.append(x)
            alone.append(xs)
    with bcs.Server(slots=3) as srv:
        ids = [srv.register(s) for s in systems]
        tickets = []
        for j in range(3):                      # round-robin arrivals
            for c in range(len(systems)):
                tickets.append((c, j, srv.submit(ids[c], seqs[c][j])))
        for c, j, t in tickets:
            st, res, lat, x = srv.wait(t)
            assert st == bcs.BCS_OK, res
            assert np.array_equal(x, alone[c][j]), (c, j)
            assert true_rel(seqs[c][j], x) <= 1e-8
            assert lat > 0
        stats = srv.stats()
    assert stats["completed"] == 12 and stats["rejected"] == 0
    assert stats["p99_ms"] >= stats["p50_ms"] > 0


def test_tight_budget_evicts_and_oversize_is_rejected():
    systems = cases()
    sizes = []
    for s_ in systems:                           # measured footprint of each case alone
        with bcs.Server(slots=1) as probe:
            cid = probe.register(s_)
            st, *_ = probe.wait(probe.submit(cid, s_))
            assert st == bcs.BCS_OK
            sizes.append(probe.stats()["resident_bytes"])
    budget = int(2.0 * max(sizes))
    assert sum(sizes) > budget                   # not every case fits at once
    with bcs.Server(budget_bytes=budget, slots=2) as srv:
        ids = [srv.register(s_) for s_ in systems]
        tickets = [(c % 4, srv.submit(ids[c % 4], systems[c % 4])) for c in range(12)]
        for c, t in tickets:
            st, res, lat, x = srv.wait(t)
            assert st == bcs.BCS_OK, res
            assert true_rel(systems[c], x) <= 1e-8
        st = srv.stats()
        assert st["resident_bytes"] <= budget
    assert st["evictions"] > 0 and st["completed"] == 12
    with bcs.Server(budget_bytes=1 << 16, slots=1) as srv:   # 64 KiB: nothing fits
        cid = srv.register(systems[0])
        st, res, lat, x = srv.wait(srv.submit(cid, systems[0]))
        assert st == bcs.BCS_REJECTED


def test_wait_with_timeout():
    system = synth.density(24, seed=5)
    with bcs.Server(slots=1) as srv:
        cid = srv.register(system)
        t = srv.submit(cid, system)
        st, res, lat, x = srv.wait(t, timeout_ms=0)
        if st == bcs.BCS_TIMEOUT:
            st, res, lat, x = srv.wait(t)
        assert st == bcs.BCS_OK and true_rel(system, x) <= 1e-8


def test_device_inputs_match_host_inputs():
    """Requests whose arrays live in device memory give the same solutions,
    bit for bit, as requests with host arrays."""
    systems = cases()[:2]
    seqs = sequences(systems, k=2)
    out = {}
    for where in ("host", "device"):
        with bcs.Server(slots=2) as srv:
            ids = [srv.register(s) for s in systems]
            tickets = []
            for c in range(len(systems)):
                for j, s_ in enumerate(seqs[c]):
                    if where == "device":
                        s_ = {k: torch.from_numpy(s_[k]).cuda() for k in ("diag", "upper", "lower", "b")}
                        torch.cuda.synchronize()
                    tickets.append((c, j, srv.submit(ids[c], s_)))
            for c, j, t in tickets:
                st, res, lat, x = srv.wait(t)
                assert st == bcs.BCS_OK, res
                out[(where, c, j)] = x if where == "host" else x.cpu().numpy()
    for c in range(len(systems)):
        for j in range(2):
            assert np.array_equal(out[("host", c, j)], out[("device", c, j)])
            assert true_rel(seqs[c][j], out[("host", c, j)]) <= 1e-8


def test_gpu_timeline_statistics():
    """The server's GPU-timeline statistics: one slot gives requests that
    never overlap (overlap share 0, at most one in flight on average);
    several slots over several cases put two or more requests' kernels in
    flight together for part of the window."""
    systems = [synth.density(14, seed=1), synth.pressure(12, seed=2), synth.density(13, 11, 9, seed=3),
               synth.pressure(11, 10, 9, seed=5)]
    dev = "cuda:0"
    data = [{k: torch.from_numpy(s[k]).to(dev) for k in ("diag", "upper", "lower", "b")} for s in systems]
    for slots in (1, 4):
        with bcs.Server(slots=slots) as srv:
            ids = [srv.register(s) for s in systems]
            # warm-up: first admission (full setup) of every case
            for t in [srv.submit(i, d) for i, d in zip(ids, data)]:
                assert srv.wait(t)[0] == bcs.BCS_OK
            srv.reset_stats()
            tickets = [srv.submit(ids[k % 4], data[k % 4]) for k in range(16)]
            for t in tickets:
                assert srv.wait(t)[0] == bcs.BCS_OK
            st = srv.stats()
        assert st["completed"] == 16 and st["window_ms"] > 0
        assert 0.0 < st["busy_frac"] <= 1.0 + 1e-9
        assert st["overlap_frac"] <= st["busy_frac"] + 1e-9
        if slots == 1:
            assert st["overlap_frac"] == 0.0 and st["mean_in_flight"] <= 1.0 + 1e-9
        else:
            assert st["overlap_frac"] > 0.0 and st["mean_in_flight"] > 1.0
        print(f"slots={slots}: window {st['window_ms']:.1f} ms busy {st['busy_frac']:.3f} "
              f"overlap {st['overlap_frac']:.3f} in flight {st['mean_in_flight']:.2f}")


def test_batching_server_results_identical():
    """With batching on, a slot solves the queued requests of several
    resident cases of the same block size together (bcs_solve_batch); each
    result equals the case's result alone, bit for bit, and batches form."""
    systems = [synth.density(10, seed=1), synth.density(12, 9, 7, seed=3), synth.density(8, seed=7),
               synth.pressure(8, seed=2), synth.density(11, 10, 6, seed=9)]
    seqs = sequences(systems)
    alone = []
    for c, system in enumerate(systems):
        with bcs.Server(slots=1) as srv:
            cid = srv.register(system)
            # the same history as below: a full setup on the system's own
            # values, then values-only resetups
            assert srv.wait(srv.submit(cid, system))[0] == bcs.BCS_OK
            xs = []
            for s in seqs[c]:
                st, res, lat, x = srv.wait(srv.submit(cid, s))
                assert st == bcs.BCS_OK, res
                xs.append(x)
            alone.append(xs)
    with bcs.Server(slots=1, batch=8) as srv:
        ids = [srv.register(s) for s in systems]
        for c in range(len(systems)):          # first admission of every case
            assert srv.wait(srv.submit(ids[c], systems[c]))[0] == bcs.BCS_OK
        srv.reset_stats()
        tickets = []
        for j in range(3):
            for c in range(len(systems)):
                tickets.append((c, j, srv.submit(ids[c], seqs[c][j])))
        for c, j, t in tickets:
            st, res, lat, x = srv.wait(t)
            assert st == bcs.BCS_OK, res
            assert np.array_equal(x, alone[c][j]), (c, j)
        stats = srv.stats()
    assert stats["batches"] >= 1 and stats["batched_requests"] >= 2
    print(f"batches {stats['batches']} serving {stats['batched_requests']} of 15 requests")


def test_failed_request_reports_its_error():
    """A request whose matrix cannot be set up (a zero diagonal block) is
    answered BCS_SINGULAR_BLOCK and leaves its message with the server; the
    case serves the next, valid request."""
    system = synth.density(6, seed=3)
    bad = dict(system)
    bad["diag"] = system["diag"].copy()
    bad["diag"][7] = 0.0
    bad["upper"] = system["upper"].copy()
    bad["lower"] = system["lower"].copy()
    with bcs.Server(slots=1) as srv:
        assert srv.last_error() == ""
        cid = srv.register(system)
        st, res, _, _ = srv.wait(srv.submit(cid, bad))
        assert st == bcs.BCS_SINGULAR_BLOCK, res
        assert "singular" in srv.last_error()
        st, res, _, x = srv.wait(srv.submit(cid, system))
        assert st == bcs.BCS_OK, res
        assert true_rel(system, x) <= 1e-8
