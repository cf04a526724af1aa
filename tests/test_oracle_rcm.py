"""Oracle pins for the reverse Cuthill-McKee locality ordering (the internal
renumbering, an analogue of Sec. 2.3's renumbering after decomposition).

Pinned against: hand-worked orderings (a 2x3 grid; two components and an
isolated cell), a relabelled path collapsing to bandwidth one, independence
from the face order, and the bandwidth of a randomly numbered 3-D grid
brought back to that of its lattice numbering."""
import numpy as np

import oracle
from paper_2403_07882_b300 import synth


def bandwidth(perm, owner, nb):
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    return int(np.abs(inv[owner] - inv[nb]).max()) if len(owner) else 0


def test_hand_worked_grid_2x3():
    # 0 1 2 / 3 4 5; start 0 (no peripheral improvement), CM 0 3 1 4 2 5
    owner = np.array([0, 1, 3, 4, 0, 1, 2], np.int32)
    nb = np.array([1, 2, 4, 5, 3, 4, 5], np.int32)
    assert list(oracle.rcm(6, owner, nb)) == [5, 2, 4, 1, 3, 0]


def test_hand_worked_components():
    # component {0, 2, 4} as a path 4 - 0 - 2, isolated 1, component {3, 5}
    owner = np.array([0, 0, 3], np.int32)
    nb = np.array([4, 2, 5], np.int32)
    # start of {0,2,4}: 0 -> last level {2, 4} -> 2 (deg 1, smaller index)
    # -> 3 levels from 2 > 2 from 0; CM from 2: 2 0 4; then 1; then 3 5
    assert list(oracle.rcm(6, owner, nb)) == [5, 3, 1, 4, 0, 2]


def test_relabelled_path_has_bandwidth_one():
    rng = np.random.default_rng(1)
    n = 50
    lab = rng.permutation(n).astype(np.int32)
    owner, nb = lab[:-1], lab[1:]
    perm = oracle.rcm(n, owner, nb)
    assert sorted(perm) == list(range(n))
    assert bandwidth(perm, owner, nb) == 1


def test_face_order_does_not_matter_and_random_grid_recovers_lattice_bandwidth():
    sys = synth.pressure(9, seed=2)       # randomly numbered 9^3 grid
    C, o, nb = sys["n_cells"], sys["owner"], sys["neighbour"]
    perm = oracle.rcm(C, o, nb)
    assert np.array_equal(np.sort(perm), np.arange(C))
    f = np.random.default_rng(3).permutation(o.size)
    assert np.array_equal(oracle.rcm(C, o[f], nb[f]), perm)
    assert bandwidth(np.arange(C, dtype=np.int32), o, nb) > 5 * 81    # random numbering
    assert bandwidth(perm, o, nb) <= 1.5 * 81                          # lattice numbering: 9^2
    assert oracle.rcm(3, np.array([0], np.int32), np.array([0], np.int32)) is None


def test_degenerate_graphs():
    assert list(oracle.rcm(1, np.zeros(0, np.int32), np.zeros(0, np.int32))) == [0]
    # no faces: every cell its own component, taken by index and reversed
    assert list(oracle.rcm(4, np.zeros(0, np.int32), np.zeros(0, np.int32))) == [3, 2, 1, 0]
    # owner > neighbour is the same edge
    a = oracle.rcm(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32))
    b = oracle.rcm(3, np.array([1, 2], np.int32), np.array([0, 1], np.int32))
    assert np.array_equal(a, b)
