"""GPU parity of the internal reverse Cuthill-McKee renumbering (reorder = 1):
the permutation equal to the CPU reference's (index work: bit-exact) on
structured, randomly numbered, unstructured and disconnected graphs; the
internal block-CSR matrix equal to the reference matrix of the relabelled
system; SpMV, solves, assembly and packing through the renumbered solver
giving results in the caller's numbering (SpMV at 1e-12, solves to 1e-8
recomputed on the CPU)."""
import numpy as np
import pytest

import oracle
from paper_2403_07882_b300 import bcs, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def islands():
    """Two grids side by side plus isolated cells (disconnected graph)."""
    a = synth.density(5, 4, 3, seed=1)
    b = synth.density(4, 3, 2, seed=2)
    Ca = a["n_cells"]
    C = Ca + b["n_cells"] + 3
    owner = np.concatenate([a["owner"], b["owner"] + Ca + 2])
    nb = np.concatenate([a["neighbour"], b["neighbour"] + Ca + 2])
    rng = np.random.default_rng(3)
    F = owner.size
    diag = np.repeat((7.0 * np.eye(5))[None], C, 0) + 0.1 * rng.standard_normal((C, 5, 5))
    return dict(n_cells=C, n_faces=F, n=5, owner=owner.astype(np.int32), neighbour=nb.astype(np.int32), diag=diag,
                upper=-np.eye(5) + 0.1 * rng.standard_normal((F, 5, 5)),
                lower=-np.eye(5) + 0.1 * rng.standard_normal((F, 5, 5)), b=rng.uniform(-1, 1, (C, 5)))


GRAPHS = [("density 9^3", lambda: synth.density(9, seed=0)),
          ("pressure 10^3 random numbering", lambda: synth.pressure(10, seed=1)),
          ("knn 8^3", lambda: synth.knn(8, seed=2)),
          ("random graph", lambda: synth.random_graph(300, 700, 3, seed=5)),
          ("islands", islands)]


def relabelled(system, perm):
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size, dtype=perm.dtype)
    return dict(system, owner=inv[system["owner"]].astype(np.int32), neighbour=inv[system["neighbour"]].astype(np.int32),
                diag=system["diag"][perm], b=system["b"][perm])


@pytest.mark.parametrize("name,gen", GRAPHS, ids=[g[0] for g in GRAPHS])
def test_permutation_matrix_spmv_and_solve(name, gen):
    system = gen()
    C = system["n_cells"]
    perm_ref = oracle.rcm(C, system["owner"], system["neighbour"])
    with bcs.Solver(system["n"], reorder=1) as s:
        s.load(system, device=DEV)
        perm = s.permutation()
        assert np.array_equal(perm, perm_ref), name
        ref = oracle.ldu_to_bsr(relabelled(system, perm_ref))
        got = s.bsr()
        assert np.array_equal(got["row_ptr"], ref["row_ptr"]) and np.array_equal(got["col"], ref["col"])
        assert np.array_equal(got["val"], ref["val"])
        x = np.random.default_rng(4).standard_normal((C, system["n"]))
        y = s.spmv(torch.from_numpy(x).to(DEV)).cpu().numpy()
        y_ref = oracle.spmv(oracle.ldu_to_bsr(system), x)
        assert np.abs(y - y_ref).max() <= 1e-12 * np.abs(y_ref).max()
        xs, st, res = s.solve(torch.from_numpy(system["b"]).to(DEV))
        assert st == bcs.BCS_OK, res
        r = system["b"] - oracle.spmv(oracle.ldu_to_bsr(system), xs.cpu().numpy())
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(system["b"])
    # host arrays, BiCGStab
    with bcs.Solver(system["n"], reorder=1, solver=bcs.BCS_BICGSTAB) as s:
        s.load(system)
        xs, st, res = s.solve(system["b"].copy())
        assert st == bcs.BCS_OK, res
        r = system["b"] - oracle.spmv(oracle.ldu_to_bsr(system), xs)
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(system["b"])


def test_assembly_and_packing_through_renumbered_solver():
    fl = synth.flow(10, 8, 6, seed=3)
    st, d_r, u_r, l_r = oracle.assemble_density(fl)
    assert st == 0
    system = dict(n_cells=fl["n_cells"], n_faces=fl["n_faces"], n=5, owner=fl["owner"], neighbour=fl["neighbour"],
                  diag=d_r, upper=u_r, lower=l_r, b=fl["b"])
    ref = oracle.ldu_to_bsr(system)
    geo = [torch.from_numpy(np.ascontiguousarray(fl[k])).to(DEV) for k in ("Q", "area", "normal", "dist")]
    with bcs.Solver(5, reorder=1) as s:
        s.set_structure(fl["n_cells"], torch.from_numpy(fl["owner"]).to(DEV),
                        torch.from_numpy(fl["neighbour"]).to(DEV))
        d, u, l = (t.cpu().numpy() for t in s.assemble_density(*geo))
        for g_, r_ in ((d, d_r), (u, u_r), (l, l_r)):
            scale = np.abs(r_).max(axis=(1, 2), keepdims=True)
            assert np.all(np.abs(g_ - r_) <= 1e-13 * scale)
        s.assemble_density(*geo, to_values=True)
        x, st, res = s.solve(torch.from_numpy(fl["b"]).to(DEV))
        assert st == bcs.BCS_OK, res
        r = fl["b"] - oracle.spmv(ref, x.cpu().numpy())
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(fl["b"]) * (1 + 1e-3)
        # the same matrix from field couplings straight into the values
        off = [0, 1, 4, 5]
        cp = [[tuple(torch.from_numpy(np.ascontiguousarray(system[k][:, off[a]:off[a + 1], off[b]:off[b + 1]])).to(DEV)
                     for k in ("diag", "upper", "lower")) for b in range(3)] for a in range(3)]
        s.pack_coefficients(cp, [1, 3, 1], to_values=True)
        assert np.array_equal(s.bsr()["val"], oracle.ldu_to_bsr(relabelled(system, s.permutation()))["val"])
