"""GPU parity of the segregated-field <-> block AoS conversions (Alg. 1 steps
1, 5 and 15): vectors and coefficients bit-exact with the CPU reference
(pure data movement) for several field splits, host and device inputs, zero
couplings; coefficients packed straight into the solver's values give the
same block-CSR matrix and the same solution bit for bit as set_values; bad
splits are refused; the 128^3 benchmark system is checked on sampled blocks."""
import numpy as np
import pytest

import oracle
from paper_2403_07882_b300 import bcs, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

SPLITS = {5: ([1, 3, 1], [2, 2, 1], [5]), 4: ([1, 3], [3, 1], [4])}


def split(system, ncomp, drop=()):
    off = oracle.field_offsets(ncomp)
    nf = len(ncomp)
    return [[None if (a, b) in drop else
             tuple(np.ascontiguousarray(system[k][:, off[a]:off[a + 1], off[b]:off[b + 1]])
                   for k in ("diag", "upper", "lower")) for b in range(nf)] for a in range(nf)]


def to_dev(coupling):
    return [[None if cp is None else tuple(torch.from_numpy(x).to(DEV) for x in cp) for cp in row]
            for row in coupling]


@pytest.mark.parametrize("gen", [lambda: synth.density(7, 5, 3, seed=1), lambda: synth.pressure(6, seed=2)],
                         ids=["density", "pressure"])
@pytest.mark.parametrize("where", ["host", "device"])
def test_pack_vector_and_coefficients_bit_exact(gen, where):
    system = gen()
    n, C, F = system["n"], system["n_cells"], system["n_faces"]
    rng = np.random.default_rng(3)
    with bcs.Solver(n) as s:
        s.set_structure(C, system["owner"], system["neighbour"])
        for ncomp in SPLITS[n]:
            fields = [rng.standard_normal(C * m) for m in ncomp]
            ref = oracle.pack_vector(fields, ncomp)
            if where == "device":
                vec = s.pack_vector([torch.from_numpy(f).to(DEV) for f in fields], ncomp).cpu().numpy()
                back = [f.cpu().numpy() for f in s.unpack_vector(torch.from_numpy(ref).to(DEV), ncomp)]
            else:
                vec = s.pack_vector(fields, ncomp)
                back = s.unpack_vector(ref, ncomp)
            assert np.array_equal(vec, ref)
            assert all(np.array_equal(x, y) for x, y in zip(back, fields))
            # coefficients, with one zero off-diagonal coupling when there are two fields or more
            drop = {(0, len(ncomp) - 1)} if len(ncomp) > 1 else set()
            cp = split(system, ncomp, drop)
            d_r, u_r, l_r = oracle.pack_coefficients(cp, ncomp, C, F)
            if where == "device":
                d, u, l = (t.cpu().numpy() for t in s.pack_coefficients(to_dev(cp), ncomp))
            else:
                d, u, l = s.pack_coefficients(cp, ncomp)
            assert np.array_equal(d, d_r) and np.array_equal(u, u_r) and np.array_equal(l, l_r)


def test_pack_into_solver_values_matches_set_values():
    system = synth.density(12, 10, 8, seed=4)
    C = system["n_cells"]
    b = torch.from_numpy(system["b"]).to(DEV)
    xs = []
    for path in ("set_values", "pack"):
        with bcs.Solver(5) as s:
            s.set_structure(C, torch.from_numpy(system["owner"]).to(DEV),
                            torch.from_numpy(system["neighbour"]).to(DEV))
            if path == "pack":
                s.pack_coefficients(to_dev(split(system, [1, 3, 1])), [1, 3, 1], to_values=True)
            else:
                s.set_values(*(torch.from_numpy(system[k]).to(DEV) for k in ("diag", "upper", "lower")))
            got = s.bsr()
            x, st, res = s.solve(b)
            assert st == bcs.BCS_OK
            xs.append((got["val"], x.cpu().numpy()))
            # values-only resetup through the packing path
            if path == "pack":
                sys2 = synth.perturb(system, np.random.default_rng(5), 0.02)
                levels = s.levels
                s.pack_coefficients(to_dev(split(sys2, [1, 3, 1])), [1, 3, 1], to_values=True)
                assert s.levels == levels
                assert np.array_equal(s.bsr()["val"], oracle.ldu_to_bsr(sys2)["val"])
    assert np.array_equal(xs[0][0], xs[1][0]) and np.array_equal(xs[0][1], xs[1][1])


def test_pack_refuses_bad_splits():
    system = synth.density(4, seed=6)
    C = system["n_cells"]
    with bcs.Solver(5) as s:
        with pytest.raises(bcs.BcsError) as e:
            s.pack_vector([np.zeros(C * 5)], [5])
        assert e.value.status == bcs.BCS_ESTATE
        s.set_structure(C, system["owner"], system["neighbour"])
        for ncomp in ([1, 3], [1, 3, 2], [0, 5], [1] * 9):
            with pytest.raises(bcs.BcsError) as e:
                s.pack_vector([np.zeros(C * max(m, 1)) for m in ncomp], ncomp)
            assert e.value.status == bcs.BCS_EINVAL, ncomp
        cp = split(system, [1, 3, 1])
        d, u, l = cp[0][1]
        cp[0][1] = (d, u, None)
        with pytest.raises(bcs.BcsError) as e:
            bcs.bcs_pack_coefficients(s.h, [1, 3, 1], cp, np.zeros((C, 5, 5)), np.zeros((s.F, 5, 5)),
                                      np.zeros((s.F, 5, 5)))
        assert e.value.status == bcs.BCS_EINVAL


def test_pack_benchmark_system_sampled():
    """128^3 density system (2.9 GB of blocks) from its nine field couplings on
    the device; sampled blocks compared with the reference."""
    system = synth.density(128, seed=2)
    C, F = system["n_cells"], system["n_faces"]
    cp = to_dev(split(system, [1, 3, 1]))
    with bcs.Solver(5) as s:
        s.set_structure(C, torch.from_numpy(system["owner"]).to(DEV), torch.from_numpy(system["neighbour"]).to(DEV))
        d, u, l = s.pack_coefficients(cp, [1, 3, 1])
        rng = np.random.default_rng(8)
        ic = torch.from_numpy(rng.integers(0, C, 4000)).to(DEV)
        jf = torch.from_numpy(rng.integers(0, F, 4000)).to(DEV)
        assert np.array_equal(d[ic].cpu().numpy(), system["diag"][ic.cpu().numpy()])
        assert np.array_equal(u[jf].cpu().numpy(), system["upper"][jf.cpu().numpy()])
        assert np.array_equal(l[jf].cpu().numpy(), system["lower"][jf.cpu().numpy()])
