"""The Python binding checks every array before a pointer reaches the
library (the C ABI receives bare pointers and cannot): dtype, element count
against the solver's block size and mesh, contiguity, one memory kind per
call. These checks run on the CPU: each call below must raise ValueError
before the library is called (the handles are stand-ins that the library
never sees)."""
import ctypes as ct

import numpy as np
import pytest

from paper_2403_07882_b300 import bcs


@pytest.fixture
def fake_handle():
    key = 0x7E57
    bcs._dims[key] = [5, 10, 20]   # n = 5, C = 10 cells, F = 20 faces
    yield ct.c_void_p(key)
    bcs._dims.pop(key, None)


def test_values_wrong_dtype_and_count(fake_handle):
    n, C, F = 5, 10, 20
    ok = (np.zeros((C, n, n)), np.zeros((F, n, n)), np.zeros((F, n, n)))
    with pytest.raises(ValueError, match="float64"):
        bcs.bcs_set_values(fake_handle, ok[0].astype(np.float32), ok[1], ok[2])
    with pytest.raises(ValueError, match="elements"):
        bcs.bcs_set_values(fake_handle, ok[0], ok[1][:-1], ok[2])
    with pytest.raises(ValueError, match="contiguous"):
        bcs.bcs_set_values(fake_handle, ok[0], np.zeros((n, n, F)).transpose(2, 0, 1), ok[2])


def test_structure_int32_and_equal_lengths(fake_handle):
    with pytest.raises(ValueError, match="int32"):
        bcs.bcs_set_structure(fake_handle, 10, np.zeros(20, np.int64), np.zeros(20, np.int64))
    with pytest.raises(ValueError, match="elements"):
        bcs.bcs_set_structure(fake_handle, 10, np.zeros(20, np.int32), np.zeros(19, np.int32))


def test_vectors_sized_by_the_mesh(fake_handle):
    with pytest.raises(ValueError, match="elements"):
        bcs.bcs_solve(fake_handle, np.zeros(49), np.zeros(50))
    with pytest.raises(ValueError, match="elements"):
        bcs.bcs_spmv(fake_handle, np.zeros(50), np.zeros(51))
    with pytest.raises(ValueError, match="float64"):
        bcs.bcs_precond_apply(fake_handle, np.zeros(50, np.float32), np.zeros(50))
    with pytest.raises(ValueError, match="elements"):
        bcs.bcs_pack_vector(fake_handle, [1, 3, 1], [np.zeros(10), np.zeros(29), np.zeros(10)], np.zeros(50))
    with pytest.raises(ValueError, match="elements"):
        bcs.bcs_assemble_density(fake_handle, np.zeros(50), np.zeros(20), np.zeros(59), np.zeros(20),
                                 bcs.bcs_flow_params())


def test_unknown_handle():
    with pytest.raises(ValueError, match="handle"):
        bcs.bcs_solve(ct.c_void_p(0xDEAD), np.zeros(5), np.zeros(5))


def test_noalloc_wrong_dtype_short_col_and_host_arrays():
    C, F = 6, 7
    i32 = lambda k: np.zeros(k, np.int32)
    with pytest.raises(ValueError, match="int32"):
        bcs.bcs_ldu_structure_noalloc(C, np.zeros(F, np.int64), i32(F), i32(C + 1), i32(C + 2 * F), i32(C),
                                      i32(F), i32(F))
    with pytest.raises(ValueError, match="elements"):
        bcs.bcs_ldu_structure_noalloc(C, i32(F), i32(F), i32(C + 1), i32(C + 2 * F - 1), i32(C), i32(F), i32(F))
    with pytest.raises(ValueError, match="elements"):
        bcs.bcs_ldu_structure_noalloc(C, i32(F), i32(F - 1), i32(C + 1), i32(C + 2 * F), i32(C), i32(F), i32(F))
    with pytest.raises(ValueError, match="device"):
        bcs.bcs_ldu_structure_noalloc(C, i32(F), i32(F), i32(C + 1), i32(C + 2 * F), i32(C), i32(F), i32(F))


def test_server_submit_sized_by_the_case():
    key = 0x5E4
    bcs._dims[(key, 3)] = [4, 8, 12]
    try:
        with pytest.raises(ValueError, match="elements"):
            bcs.bcs_server_submit(ct.c_void_p(key), 3, np.zeros((8, 4, 4)), np.zeros((12, 4, 4)),
                                  np.zeros((11, 4, 4)), np.zeros((8, 4)), np.zeros((8, 4)))
        with pytest.raises(ValueError, match="registered"):
            bcs.bcs_server_submit(ct.c_void_p(key), 4, np.zeros((8, 4, 4)), np.zeros((12, 4, 4)),
                                  np.zeros((12, 4, 4)), np.zeros((8, 4)), np.zeros((8, 4)))
    finally:
        bcs._dims.pop((key, 3), None)
