"""Oracle pins for the segregated-field <-> block AoS conversions (Alg. 1
steps 1, 5 and 15): a hand-written two-cell example of each, round trips,
and the coupled density system rebuilt from its field couplings."""
import numpy as np

import oracle
from paper_2403_07882_b300 import synth


def test_pack_vector_hand_example():
    # fields rho (scalar), rhoU (vector, [cell][3]), rhoE (scalar), two cells
    rho = np.array([1.0, 2.0])
    rhoU = np.array([10.0, 11.0, 12.0, 20.0, 21.0, 22.0])
    rhoE = np.array([100.0, 200.0])
    out = oracle.pack_vector([rho, rhoU, rhoE], [1, 3, 1])
    assert np.array_equal(out, [[1, 10, 11, 12, 100], [2, 20, 21, 22, 200]])
    back = oracle.unpack_vector(out, [1, 3, 1])
    assert all(np.array_equal(x, y) for x, y in zip(back, [rho, rhoU, rhoE]))


def test_pack_coefficients_hand_example():
    # p (scalar) and U (vector): couplings pp, pU (1x3), Up (3x1), UU (3x3)
    C, F = 2, 1
    pp = (np.array([1.0, 2.0]), np.array([3.0]), np.array([4.0]))
    pU = (np.arange(6.0).reshape(2, 1, 3) + 10, np.array([[[20.0, 21, 22]]]), np.array([[[30.0, 31, 32]]]))
    UU = None
    Up = (np.arange(6.0).reshape(2, 3, 1) + 40, np.array([[[50.0], [51], [52]]]), np.array([[[60.0], [61], [62]]]))
    d, u, l = oracle.pack_coefficients([[pp, pU], [Up, UU]], [1, 3], C, F)
    assert np.array_equal(d[0], [[1, 10, 11, 12], [40, 0, 0, 0], [41, 0, 0, 0], [42, 0, 0, 0]])
    assert np.array_equal(d[1], [[2, 13, 14, 15], [43, 0, 0, 0], [44, 0, 0, 0], [45, 0, 0, 0]])
    assert np.array_equal(u[0], [[3, 20, 21, 22], [50, 0, 0, 0], [51, 0, 0, 0], [52, 0, 0, 0]])
    assert np.array_equal(l[0], [[4, 30, 31, 32], [60, 0, 0, 0], [61, 0, 0, 0], [62, 0, 0, 0]])


def split_couplings(system, ncomp):
    off = oracle.field_offsets(ncomp)
    return [[tuple(np.ascontiguousarray(system[k][:, off[a]:off[a + 1], off[b]:off[b + 1]])
                   for k in ("diag", "upper", "lower")) for b in range(len(ncomp))] for a in range(len(ncomp))]


def test_round_trips():
    rng = np.random.default_rng(3)
    for ncomp in ([1, 3, 1], [1, 3], [2, 2, 1], [5]):
        C = 7
        fields = [rng.standard_normal(C * m) for m in ncomp]
        vec = oracle.pack_vector(fields, ncomp)
        assert all(np.array_equal(x, y) for x, y in zip(oracle.unpack_vector(vec, ncomp), fields))
    system = synth.density(4, 3, 2, seed=1)
    d, u, l = oracle.pack_coefficients(split_couplings(system, [1, 3, 1]), [1, 3, 1],
                                       system["n_cells"], system["n_faces"])
    assert np.array_equal(d, system["diag"]) and np.array_equal(u, system["upper"])
    assert np.array_equal(l, system["lower"])


def test_single_field_is_identity_and_all_zero_couplings():
    rng = np.random.default_rng(4)
    C, F = 5, 4
    v = rng.standard_normal(C * 4)
    assert np.array_equal(oracle.pack_vector([v], [4]), v.reshape(C, 4))
    d, u, l = oracle.pack_coefficients([[None, None], [None, None]], [2, 2], C, F)
    assert not d.any() and not u.any() and not l.any() and d.shape == (C, 4, 4)
