"""Caller-supplied device allocator (bcs_config.alloc / release): with
PyTorch's caching allocator every solver buffer shows up in PyTorch's memory
statistics while the solver lives and is returned when it is destroyed;
results equal those of the default stream-ordered allocator bit for bit; an
allocator that runs dry makes the upload fail with BCS_ENOMEM and leaves
nothing behind."""
import numpy as np
import pytest

from paper_2403_07882_b300 import bcs, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_torch_allocator_accounting_and_identical_results():
    system = synth.density(16, seed=0)
    d = {k: torch.from_numpy(system[k]).to(DEV) for k in ("owner", "neighbour", "diag", "upper", "lower", "b")}
    xs = [torch.zeros_like(d["b"]) for _ in range(2)]
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    with bcs.Solver(5, allocator="torch") as s:
        s.set_structure(system["n_cells"], d["owner"], d["neighbour"])
        s.set_values(d["diag"], d["upper"], d["lower"])
        _, st, res = s.solve(d["b"], xs[0])
        assert st == bcs.BCS_OK, res
        torch.cuda.synchronize()
        held = torch.cuda.memory_allocated() - base
        assert held >= bcs.bcs_device_bytes(s.h) > 0
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base
    with bcs.Solver(5) as s:
        s.set_structure(system["n_cells"], d["owner"], d["neighbour"])
        s.set_values(d["diag"], d["upper"], d["lower"])
        _, st, res = s.solve(d["b"], xs[1])
        assert st == bcs.BCS_OK
    assert torch.equal(xs[0], xs[1])


def test_allocator_running_dry_gives_enomem():
    system = synth.density(8, seed=1)
    budget = [40]  # allocations granted before the allocator refuses

    def _alloc(nbytes, stream, user):
        if budget[0] <= 0:
            return None
        budget[0] -= 1
        return torch.cuda.caching_allocator_alloc(nbytes, stream=stream or 0)

    def _release(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    cbs = (bcs.ALLOC_FN(_alloc), bcs.RELEASE_FN(_release))
    cfg = bcs.bcs_config_default()
    cfg.alloc, cfg.release = cbs
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    h = bcs.bcs_create(5, cfg)
    try:
        with pytest.raises(bcs.BcsError) as e:
            bcs.bcs_set_structure(h, system["n_cells"], system["owner"], system["neighbour"])
            bcs.bcs_set_values(h, system["diag"], system["upper"], system["lower"])
        assert e.value.status == bcs.BCS_ENOMEM
    finally:
        bcs.bcs_destroy(h)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base


def test_misaligned_allocator_memory_is_refused():
    """Memory that is not 256-byte aligned is handed back unused and the
    upload fails with BCS_ENOMEM (the kernels' vector accesses rely on it)."""
    system = synth.density(4, seed=2)

    def _alloc(nbytes, stream, user):
        return torch.cuda.caching_allocator_alloc(nbytes + 64, stream=stream or 0) + 16

    def _release(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr - 16)

    cbs = (bcs.ALLOC_FN(_alloc), bcs.RELEASE_FN(_release))
    cfg = bcs.bcs_config_default()
    cfg.alloc, cfg.release = cbs
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    with pytest.raises(bcs.BcsError) as e:
        h = bcs.bcs_create(5, cfg)
        try:
            bcs.bcs_set_structure(h, system["n_cells"], system["owner"], system["neighbour"])
        finally:
            bcs.bcs_destroy(h)
    assert e.value.status == bcs.BCS_ENOMEM
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base
