"""The allocation-free structure build, checked against bcs_set_structure.

bcs_ldu_structure_noalloc serves callers that may not let the library
allocate device memory (a fixed memory budget reserved up front, or a ban on
cudaMalloc after start-up because it synchronises the device). It keeps its
scratch in a fixed array inside the library, shared by every call, so this
test runs two builds in a row (different meshes, the second smaller than the
first) to show that the leftovers of one call do not leak into the next.
This file is collected last on purpose.
"""
import ctypes as ct

import numpy as np
import pytest

from paper_2403_07882_b300 import bcs, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def reference_structure(system):
    with bcs.Solver(system["n"]) as s:
        s.set_structure(system["n_cells"], torch.from_numpy(system["owner"]).to(DEV),
                        torch.from_numpy(system["neighbour"]).to(DEV))
        return s.bsr(values=False)


def noalloc_structure(system):
    C, F = system["n_cells"], system["n_faces"]
    i32 = dict(dtype=torch.int32, device=DEV)
    out = dict(row_ptr=torch.full((C + 1,), -7, **i32), col=torch.full((C + 2 * F,), -7, **i32),
               pos_diag=torch.full((C,), -7, **i32), pos_up=torch.full((F,), -7, **i32),
               pos_lo=torch.full((F,), -7, **i32))
    st, msg = bcs.bcs_ldu_structure_noalloc(C, torch.from_numpy(system["owner"]).to(DEV),
                                            torch.from_numpy(system["neighbour"]).to(DEV), out["row_ptr"],
                                            out["col"], out["pos_diag"], out["pos_up"], out["pos_lo"])
    assert st == bcs.BCS_OK, msg
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_two_calls_in_a_row_match_set_structure():
    for system in (synth.pressure(24, seed=3), synth.density(10, 9, 7, seed=1)):
        ref = reference_structure(system)
        got = noalloc_structure(system)
        for key in ("row_ptr", "col", "pos_diag", "pos_up", "pos_lo"):
            assert np.array_equal(got[key], ref[key]), key


def random_structure(C, F, seed):
    """Random simple graph with C cells and about F faces (vectorised draw,
    repeated pairs dropped), owner < neighbour, faces in random order."""
    rng = np.random.default_rng(seed)
    a, b = rng.integers(0, C, F), rng.integers(0, C, F)
    keep = a != b
    lo, hi = np.minimum(a[keep], b[keep]), np.maximum(a[keep], b[keep])
    key = np.unique(lo.astype(np.int64) * C + hi)
    rng.shuffle(key)
    return dict(n=1, n_cells=C, n_faces=key.size, owner=(key // C).astype(np.int32),
                neighbour=(key % C).astype(np.int32))


def test_full_limit_matches_set_structure():
    """Exactly 1048576 cells: 1024 scan tiles, every thread of the tile-sum
    scan in use and the tile-sum area of the fixed array full."""
    system = random_structure(1 << 20, 3 << 20, seed=21)
    ref = reference_structure(system)
    got = noalloc_structure(system)
    for key in ("row_ptr", "col", "pos_diag", "pos_up", "pos_lo"):
        assert np.array_equal(got[key], ref[key]), key


def test_repeated_face_rejected():
    """A face given twice, also with owner and neighbour swapped, is a
    repeated cell pair: BCS_EINVAL, and the next valid call is unaffected."""
    i32 = dict(dtype=torch.int32, device=DEV)
    for owner, nb in (([0, 1, 0], [1, 2, 1]), ([0, 1, 2], [1, 2, 1])):
        C, F = 3, len(owner)
        out = [torch.zeros(k, **i32) for k in (C + 1, C + 2 * F, C, F, F)]
        st, msg = bcs.bcs_ldu_structure_noalloc(C, torch.tensor(owner, **i32), torch.tensor(nb, **i32), *out)
        assert st == bcs.BCS_EINVAL and "repeated" in msg, msg
    system = synth.random_graph(150, 400, 2, seed=9)
    ref = reference_structure(system)
    got = noalloc_structure(system)
    assert all(np.array_equal(got[k], ref[k]) for k in ("row_ptr", "col", "pos_diag", "pos_up", "pos_lo"))


def test_host_arrays_rejected_through_the_c_abi():
    """Host (numpy) arrays handed straight to the C entry point are refused
    with BCS_EINVAL before anything is launched; the outputs stay as they
    were."""
    C, F = 4, 3
    owner = np.array([0, 1, 2], np.int32)
    nb = np.array([1, 2, 3], np.int32)
    outs = [np.full(k, -7, np.int32) for k in (C + 1, C + 2 * F, C, F, F)]
    buf = ct.create_string_buffer(256)
    st = bcs.lib().bcs_ldu_structure_noalloc(C, F, owner.ctypes.data, nb.ctypes.data,
                                             *(o.ctypes.data for o in outs), None, buf, 256)
    assert st == bcs.BCS_EINVAL and "device memory" in buf.value.decode()
    assert all(np.all(o == -7) for o in outs)
    # one host array among device arrays is refused too
    i32 = dict(dtype=torch.int32, device=DEV)
    dev_outs = [torch.zeros(k, **i32) for k in (C + 1, C + 2 * F, C, F, F)]
    dev_owner = torch.tensor(owner, **i32)
    st = bcs.lib().bcs_ldu_structure_noalloc(C, F, dev_owner.data_ptr(), nb.ctypes.data,
                                             *(o.data_ptr() for o in dev_outs), None, buf, 256)
    assert st == bcs.BCS_EINVAL


def test_rejects_oversize_and_bad_faces():
    i32 = dict(dtype=torch.int32, device=DEV)
    big = (1 << 20) + 1
    z = torch.zeros(1, **i32)
    st, msg = bcs.bcs_ldu_structure_noalloc(big, z, z, z, z, z, z, z)
    assert st == bcs.BCS_EINVAL and "1048576" in msg
    owner = torch.tensor([0, 1], **i32)
    nb = torch.tensor([1, 5], **i32)   # cell 5 does not exist
    rp, col, pd = torch.zeros(4, **i32), torch.zeros(7, **i32), torch.zeros(3, **i32)
    pu, pl = torch.zeros(2, **i32), torch.zeros(2, **i32)
    st, msg = bcs.bcs_ldu_structure_noalloc(3, owner, nb, rp, col, pd, pu, pl)
    assert st == bcs.BCS_EINVAL and "out of range" in msg
    # a valid call right after a rejected one still matches the reference
    system = synth.random_graph(200, 500, 2, seed=8)
    ref = reference_structure(system)
    got = noalloc_structure(system)
    assert all(np.array_equal(got[k], ref[k]) for k in ("row_ptr", "col", "pos_diag", "pos_up", "pos_lo"))
