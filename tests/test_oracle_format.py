"""Oracle pins for the LDU addressing, the LDU -> block-CSR map and the BSR SpMV.

Pinned against: a hand-worked LDU example (golden), the definition of Eq. 1
assembled densely by brute force, bit-exact round trips, numpy's dense matvec,
and special cases (identity blocks, a single cell).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2403_07882_b300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def dense_from_ldu(sys):
    """Eq. 1 assembled entry by entry: the plain definition of A."""
    C, n = sys["n_cells"], sys["n"]
    A = np.zeros((C * n, C * n))
    for i in range(C):
        A[i * n:(i + 1) * n, i * n:(i + 1) * n] = sys["diag"][i]
    for f in range(sys["n_faces"]):
        o, m = sys["owner"][f], sys["neighbour"][f]
        A[o * n:(o + 1) * n, m * n:(m + 1) * n] = sys["upper"][f]
        A[m * n:(m + 1) * n, o * n:(o + 1) * n] = sys["lower"][f]
    return A


def dense_from_bsr(bsr):
    rows, n = bsr["rows"], bsr["n"]
    cols = rows if "cols" not in bsr else bsr["cols"]
    A = np.zeros((rows * n, cols * n))
    for i in range(rows):
        for k in range(bsr["row_ptr"][i], bsr["row_ptr"][i + 1]):
            j = bsr["col"][k]
            A[i * n:(i + 1) * n, j * n:(j + 1) * n] = bsr["val"][k]
    return A


def tiny_systems():
    yield synth.density(2, 2, 2, seed=5)
    yield synth.density(3, 2, 1, seed=6)
    yield synth.pressure(3, 2, 2, seed=7)
    for s in range(4):
        yield synth.random_graph(12, 20, 1 + s, seed=s)


def test_golden_chain():
    g = json.load(open(os.path.join(GOLD, "ldu_chain3.json")))
    for case in (g, g["reversed_face_case"]):
        sys = dict(n_cells=case["cells"], n_faces=len(case["owner"]), n=1,
                   owner=np.array(case["owner"], np.int32), neighbour=np.array(case["neighbour"], np.int32),
                   diag=np.ones((case["cells"], 1, 1)), upper=np.full((len(case["owner"]), 1, 1), 2.0),
                   lower=np.full((len(case["owner"]), 1, 1), 3.0))
        b = oracle.ldu_to_bsr(sys)
        for key in ("row_ptr", "col", "pos_diag", "pos_up", "pos_lo"):
            assert b[key].tolist() == case[key], key


@pytest.mark.parametrize("owner,neighbour,C", [
    ([0, 1], [1, 3], 3),        # out of range
    ([0, 1], [1, 1], 3),        # self face
    ([0, 1, 1], [1, 2, 0], 3),  # the same pair twice (reversed)
    ([0, 0], [1, 1], 2),        # exact duplicate
    ([-1], [0], 2),             # negative
])
def test_check_rejects(owner, neighbour, C):
    assert oracle.ldu_check(C, owner, neighbour) == 1


def test_check_rejects_no_cells():
    assert oracle.ldu_check(0, [], []) == 1


@pytest.mark.parametrize("k", range(7))
def test_bsr_equals_definition(k):
    sys = list(tiny_systems())[k]
    b = oracle.ldu_to_bsr(sys)
    assert np.array_equal(dense_from_bsr(b), dense_from_ldu(sys))
    rp, col = b["row_ptr"], b["col"]
    for i in range(b["rows"]):
        cols = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(cols) > 0)
        assert i in cols
    deg = np.bincount(np.concatenate([sys["owner"], sys["neighbour"]]), minlength=sys["n_cells"])
    assert np.array_equal(np.diff(rp), deg + 1)


@pytest.mark.parametrize("k", range(7))
def test_round_trip_bit_exact(k):
    sys = list(tiny_systems())[k]
    b = oracle.ldu_to_bsr(sys)
    d, u, lo = oracle.bsr_to_ldu(b, sys["n_faces"])
    assert np.array_equal(d, sys["diag"]) and np.array_equal(u, sys["upper"]) and np.array_equal(lo, sys["lower"])


def test_round_trip_c1():
    sys = synth.density(16, seed=0)
    b = oracle.ldu_to_bsr(sys)
    d, u, lo = oracle.bsr_to_ldu(b, sys["n_faces"])
    assert np.array_equal(d, sys["diag"]) and np.array_equal(u, sys["upper"]) and np.array_equal(lo, sys["lower"])
    assert b["row_ptr"][-1] == 27136


@pytest.mark.parametrize("k", range(7))
def test_spmv_vs_dense(k):
    sys = list(tiny_systems())[k]
    b = oracle.ldu_to_bsr(sys)
    x = np.random.default_rng(k).standard_normal((b["rows"], b["n"]))
    y = oracle.spmv(b, x)
    ref = dense_from_ldu(sys) @ x.ravel()
    scale = np.abs(dense_from_ldu(sys)) @ np.abs(x.ravel())
    assert np.all(np.abs(y.ravel() - ref) <= 1e-14 * scale + 1e-300)


def test_spmv_identity_blocks_exact():
    sys = synth.density(3, 3, 2, seed=1)
    n = sys["n"]
    sys["diag"][:] = np.eye(n)
    sys["upper"][:] = 0.0
    sys["lower"][:] = 0.0
    b = oracle.ldu_to_bsr(sys)
    x = np.random.default_rng(0).standard_normal((b["rows"], n))
    assert np.array_equal(oracle.spmv(b, x), x)


def test_spmv_single_cell():
    rng = np.random.default_rng(3)
    D = rng.standard_normal((1, 4, 4))
    sys = dict(n_cells=1, n_faces=0, n=4, owner=np.zeros(0, np.int32), neighbour=np.zeros(0, np.int32),
               diag=D, upper=np.zeros((0, 4, 4)), lower=np.zeros((0, 4, 4)))
    b = oracle.ldu_to_bsr(sys)
    x = rng.standard_normal((1, 4))
    y = oracle.spmv(b, x)
    assert np.allclose(y[0], D[0] @ x[0], rtol=1e-15, atol=1e-15)


def test_block_norms_match_frobenius():
    rng = np.random.default_rng(11)
    v = rng.standard_normal((50, 5, 5))
    nrm = oracle.block_norms(v)
    assert np.allclose(nrm, np.linalg.norm(v, axis=(1, 2)), rtol=2e-15, atol=0)
    one = np.zeros((1, 3, 3))
    one[0, 1, 2] = -7.25
    assert oracle.block_norms(one)[0] == 7.25
