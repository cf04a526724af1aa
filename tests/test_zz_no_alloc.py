"""The allocation-free structure build, checked against bcs_set_structure.

bcs_ldu_structure_noalloc serves callers that may not let the library
allocate device memory (a fixed memory budget reserved up front, or a ban on
cudaMalloc after start-up because it synchronises the device). It keeps its
scratch in a fixed array inside the library, shared by every call, so this
test runs two builds in a row (different meshes, the second smaller than the
first) to show that the leftovers of one call do not leak into the next.
This file is collected last on purpose.
"""
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
