"""GPU parity of the density-based assembly (Sec. 2.1, Eqs. approxJac1 /
approxJac2 with the pseudo-time term): LDU blocks from host and device
inputs, and blocks written straight into the solver's block-CSR values, equal
to the CPU reference within 1e-13 of each block's largest entry (the GPU sums
a cell's own Jacobians through the linearity of J in n, the reference face by
face); assembled systems solve to 1e-8 (true residual recomputed on the CPU)
after a full setup and after a values-only resetup; bad inputs are refused;
the 128^3 benchmark mesh is checked on sampled cells and faces."""
import numpy as np
import pytest

import oracle
from paper_2403_07882_b300 import bcs, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-13


def ref_ldu(fl, **prm):
    st, d, u, l = oracle.assemble_density(fl, **prm)
    assert st == 0
    return d, u, l


def close_blocks(g, r):
    scale = np.abs(r).max(axis=(1, 2), keepdims=True)
    return np.all(np.abs(g - r) <= TOL * scale)


def geometry(fl, device=None):
    keys = ("Q", "area", "normal", "dist")
    if device is None:
        return [np.ascontiguousarray(fl[k]) for k in keys]
    return [torch.from_numpy(np.ascontiguousarray(fl[k])).to(device) for k in keys]


CASES = [("6x5x4", lambda: synth.flow(6, 5, 4, seed=1), {}),
         ("6x5x4 skewed", lambda: synth.flow(6, 5, 4, seed=2, skew=True), dict(cfl=3.0, mu=0.02)),
         ("20^3", lambda: synth.flow(20, seed=3), {}),
         ("17x9x33 skewed", lambda: synth.flow(17, 9, 33, seed=4, skew=True), dict(cfl=50.0))]


@pytest.mark.parametrize("name,gen,prm", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("where", ["host", "device"])
def test_assembly_ldu_parity(name, gen, prm, where):
    fl = gen()
    d_r, u_r, l_r = ref_ldu(fl, **prm)
    with bcs.Solver(5) as s:
        if where == "host":
            s.set_structure(fl["n_cells"], fl["owner"], fl["neighbour"])
            d, u, l = s.assemble_density(*geometry(fl), **prm)
        else:
            s.set_structure(fl["n_cells"], torch.from_numpy(fl["owner"]).to(DEV),
                            torch.from_numpy(fl["neighbour"]).to(DEV))
            d, u, l = (t.cpu().numpy() for t in s.assemble_density(*geometry(fl, DEV), **prm))
    assert close_blocks(d, d_r) and close_blocks(u, u_r) and close_blocks(l, l_r), name


@pytest.mark.parametrize("solver", [bcs.BCS_FGMRES, bcs.BCS_BICGSTAB], ids=["fgmres", "bicgstab"])
def test_assembly_into_solver_values_and_solve(solver):
    fl = synth.flow(16, 12, 10, seed=5)
    d_r, u_r, l_r = ref_ldu(fl)
    ref = oracle.ldu_to_bsr(dict(n_cells=fl["n_cells"], n_faces=fl["n_faces"], n=5, owner=fl["owner"],
                                 neighbour=fl["neighbour"], diag=d_r, upper=u_r, lower=l_r, b=fl["b"]))
    with bcs.Solver(5, solver=solver) as s:
        s.set_structure(fl["n_cells"], torch.from_numpy(fl["owner"]).to(DEV),
                        torch.from_numpy(fl["neighbour"]).to(DEV))
        geo = geometry(fl, DEV)
        s.assemble_density(*geo, to_values=True)
        got = s.bsr()
        assert np.array_equal(got["row_ptr"], ref["row_ptr"]) and np.array_equal(got["col"], ref["col"])
        assert close_blocks(got["val"], ref["val"])
        b = torch.from_numpy(fl["b"]).to(DEV)
        x, st, res = s.solve(b)
        assert st == bcs.BCS_OK, res
        r = fl["b"] - oracle.spmv(ref, x.cpu().numpy())
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(fl["b"]) * (1 + 1e-3)
        # next nonlinear iteration: new state, values-only resetup
        fl2 = dict(fl, Q=fl["Q"] * (1 + 0.01 * np.random.default_rng(1).uniform(-1, 1, fl["Q"].shape)))
        d2, u2, l2 = ref_ldu(fl2)
        ref2 = oracle.ldu_to_bsr(dict(ref, n_cells=fl["n_cells"], n_faces=fl["n_faces"], owner=fl["owner"],
                                      neighbour=fl["neighbour"], diag=d2, upper=u2, lower=l2))
        geo[0] = torch.from_numpy(fl2["Q"]).to(DEV)
        levels = s.levels
        s.assemble_density(*geo, to_values=True)
        assert s.levels == levels
        assert close_blocks(s.bsr()["val"], ref2["val"])
        x, st, res = s.solve(b)
        assert st == bcs.BCS_OK, res
        r = fl["b"] - oracle.spmv(ref2, x.cpu().numpy())
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(fl["b"]) * (1 + 1e-3)


def test_assembly_refuses_bad_input():
    fl = synth.flow(4, seed=6)
    with bcs.Solver(5) as s:
        with pytest.raises(bcs.BcsError) as e:
            s.assemble_density(*geometry(fl))
        assert e.value.status == bcs.BCS_ESTATE
        s.set_structure(fl["n_cells"], fl["owner"], fl["neighbour"])
        Q, area, normal, dist = geometry(fl)
        for bad in ({"Q": (5, 0, -1.0)}, {"Q": (9, 4, 0.0)}, {"dist": (3, None, 0.0)}, {"area": (2, None, -1.0)}):
            (k, (i, j, v)), = bad.items()
            arrs = dict(Q=Q.copy(), area=area.copy(), normal=normal, dist=dist.copy())
            if j is None:
                arrs[k][i] = v
            else:
                arrs[k][i, j] = v
            with pytest.raises(bcs.BcsError) as e:
                s.assemble_density(arrs["Q"], arrs["area"], arrs["normal"], arrs["dist"])
            assert e.value.status == bcs.BCS_EINVAL, bad
        for prm in (dict(cfl=0.0), dict(gamma=1.0), dict(prandtl=-1.0), dict(mu=float("nan"))):
            with pytest.raises(bcs.BcsError) as e:
                s.assemble_density(Q, area, normal, dist, **prm)
            assert e.value.status == bcs.BCS_EINVAL, prm
        # writing the solver's values with a bad state leaves it without values
        badQ = Q.copy()
        badQ[0, 0] = -1.0
        with pytest.raises(bcs.BcsError):
            s.assemble_density(badQ, area, normal, dist, to_values=True)
        with pytest.raises(bcs.BcsError) as e:
            s.solve(np.ones((fl["n_cells"], 5)))
        assert e.value.status == bcs.BCS_ESTATE
        s.assemble_density(Q, area, normal, dist, to_values=True)
        x, st, res = s.solve(fl["b"].copy())
        assert st == bcs.BCS_OK
    with bcs.Solver(4) as s:
        s.set_structure(fl["n_cells"], fl["owner"], fl["neighbour"])
        with pytest.raises(bcs.BcsError) as e:
            s.assemble_density(Q, area, normal, dist)
        assert e.value.status == bcs.BCS_EINVAL


def submesh(fl, cells):
    """The faces touching `cells` and every cell they touch, renumbered."""
    o, nb = fl["owner"], fl["neighbour"]
    sel = np.isin(o, cells) | np.isin(nb, cells)
    faces = np.nonzero(sel)[0]
    keep = np.unique(np.concatenate([cells, o[faces], nb[faces]]))
    new = np.full(fl["n_cells"], -1, np.int64)
    new[keep] = np.arange(keep.size)
    sub = dict(n_cells=int(keep.size), n_faces=int(faces.size), owner=new[o[faces]].astype(np.int32),
               neighbour=new[nb[faces]].astype(np.int32), Q=fl["Q"][keep], area=fl["area"][faces],
               normal=fl["normal"][faces], dist=fl["dist"][faces])
    return sub, faces, new[cells]


def test_assembly_benchmark_mesh_sampled():
    """128^3 (2.1 M cells, 6.2 M faces), the benchmark's mesh: sampled cells'
    diagonal blocks and every block of their faces against the reference
    evaluated on the sub-mesh around them."""
    fl = synth.flow(128, seed=5)
    rng = np.random.default_rng(7)
    cells = np.unique(rng.integers(0, fl["n_cells"], 2000))
    cells = np.unique(np.concatenate([cells, [0, fl["n_cells"] - 1]]))
    sub, faces, local = submesh(fl, cells)
    d_r, u_r, l_r = ref_ldu(sub)
    with bcs.Solver(5) as s:
        s.set_structure(fl["n_cells"], torch.from_numpy(fl["owner"]).to(DEV),
                        torch.from_numpy(fl["neighbour"]).to(DEV))
        d, u, l = s.assemble_density(*geometry(fl, DEV))
        idx_c = torch.from_numpy(cells).to(DEV)
        idx_f = torch.from_numpy(faces).to(DEV)
        d, u, l = d[idx_c].cpu().numpy(), u[idx_f].cpu().numpy(), l[idx_f].cpu().numpy()
    assert close_blocks(d, d_r[local]) and close_blocks(u, u_r) and close_blocks(l, l_r)
