"""CPU checks of the C ABI boundary: the library builds, loads without a
GPU, and exports every function include/bcs.h declares; calls that need no
device reject bad arguments."""
import ctypes as ct
import os
import re

import pytest

from paper_2403_07882_b300 import bcs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_names():
    text = open(os.path.join(ROOT, "include", "bcs.h")).read()
    return sorted(set(re.findall(r"^BCS_API\s+[\w\s\*]+?\b(bcs_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2403_07882_b300 import build
    build.build()
    return bcs.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_names()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(bcs.exported_names()) == names


def test_config_default_and_null_checks(lib):
    cfg = bcs.bcs_config_default()
    assert cfg.restart == 30 and cfg.tol == 1e-8 and cfg.pmode == bcs.BCS_P_TENTATIVE
    assert cfg.precision == bcs.BCS_PREC_FP32
    assert lib.bcs_config_default(None) == bcs.BCS_EINVAL
    assert lib.bcs_destroy(None) == bcs.BCS_OK
    assert lib.bcs_create(None, 5, None, None) == bcs.BCS_EINVAL
    h = ct.c_void_p()
    assert lib.bcs_create(ct.byref(h), 9, None, None) == bcs.BCS_EINVAL   # block size out of range
    bad = bcs.bcs_config_default(restart=0)
    assert lib.bcs_create(ct.byref(h), 5, ct.byref(bad), None) == bcs.BCS_EINVAL
    half = bcs.bcs_config_default()
    half.alloc = bcs.ALLOC_FN(lambda nbytes, stream, user: None)   # alloc without release
    assert lib.bcs_create(ct.byref(h), 5, ct.byref(half), None) == bcs.BCS_EINVAL
    assert lib.bcs_solve(None, None, None, 0, None) == bcs.BCS_EINVAL
    assert lib.bcs_num_levels(None) == 0
    assert lib.bcs_last_error(None) == b"null solver"


def test_kernel_kind_names(lib):
    names = [bcs.bcs_kernel_kind_name(k) for k in range(bcs.NUM_KERNEL_KINDS)]
    assert names[1] == "spmv_fp64" and names[2] == "jacobi_sweep"
    assert names[-1] == ""


def test_struct_layouts_match_header():
    text = open(os.path.join(ROOT, "include", "bcs.h")).read()
    body = re.search(r"typedef struct bcs_config \{(.*?)\} bcs_config;", text, re.S).group(1)
    fields = re.findall(r"^\s*(?:int|double|void\s*\*)\s+([\w, ]+);|^\s*void\s*\*?\s*\(\*(\w+)\)", body, re.M)
    names = [f.strip() for a, b in fields for f in (a.split(",") if a else [b])]
    assert names == [f for f, _ in bcs.bcs_config._fields_]
    assert names[-3:] == ["alloc", "release", "alloc_user"]
    body = re.search(r"typedef struct bcs_result \{(.*?)\} bcs_result;", text, re.S).group(1)
    names = [f.strip() for group in re.findall(r"^\s*(?:int|double)\s+([\w, ]+);", body, re.M)
             for f in group.split(",")]
    assert names == [f for f, _ in bcs.bcs_result._fields_]


def test_server_argument_checks(lib):
    h = ct.c_void_p()
    assert lib.bcs_server_create(ct.byref(h), 0, 0, None) == bcs.BCS_EINVAL    # no slots
    assert lib.bcs_server_create(None, 0, 2, None) == bcs.BCS_EINVAL
    assert lib.bcs_server_destroy(None) == bcs.BCS_OK
    cid = ct.c_int()
    assert lib.bcs_server_register_case(None, 5, 10, 0, None, None, ct.byref(cid)) == bcs.BCS_EINVAL
    t = ct.c_int64()
    assert lib.bcs_server_submit(None, 0, None, None, None, None, None, bcs.BCS_MEM_HOST,
                                 ct.byref(t)) == bcs.BCS_EINVAL
