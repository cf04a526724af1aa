"""Seeded synthetic block-coupled systems in OpenFOAM LDU face form.

This module only draws inputs; it holds none of the solver's arithmetic and is
the one module shared by the CPU oracle tests and the CUDA path.

A system is a dict with
    n_cells C, n_faces F, block n,
    owner[F], neighbour[F]   int32, owner < neighbour, faces sorted by
                             (owner, neighbour) (upper-triangular face order),
    diag[C, n, n]            block A_ii of Eq. 1,
    upper[F, n, n]           block (row owner, column neighbour),
    lower[F, n, n]           block (row neighbour, column owner),
    b[C, n]                  right-hand side,
all float64, row-major, C-contiguous ("block AoS", Sec. 2.3).

Workloads (the paper's CRM and DrivAer meshes are not available; these stand
in for them with the block structure of Sec. 2.1 and Sec. 2.2):
    density(nx, ny, nz, seed)   5x5 density-based system on a hex grid
    pressure(nx, ny, nz, seed)  4x4 (p, Ux, Uy, Uz) pressure-based system with a
                                randomly permuted cell numbering
    knn(npts, seed)             unstructured: jittered lattice, k-nearest
                                neighbour faces, 5x5 blocks as density()
    perturb(sys, rng, eps)      values-only change on a fixed sparsity
    flow(nx, ny, nz, seed)      cell flow state Q and face geometry of a hex
                                grid, the input of the density-based assembly
"""
import numpy as np


def _hex_faces(nx, ny, nz):
    """Internal faces of an nx*ny*nz hex grid, cell id i + nx*(j + ny*k).

    Returns (lo, hi, axis) with lo < hi in lattice numbering.
    """
    idx = np.arange(nx * ny * nz, dtype=np.int64).reshape(nz, ny, nx)
    los, his, axes = [], [], []
    for axis, (a, b) in enumerate((
            (idx[:, :, :-1], idx[:, :, 1:]),
            (idx[:, :-1, :], idx[:, 1:, :]),
            (idx[:-1, :, :], idx[1:, :, :]))):
        los.append(a.ravel())
        his.append(b.ravel())
        axes.append(np.full(a.size, axis, dtype=np.int8))
    return np.concatenate(los), np.concatenate(his), np.concatenate(axes)


def _sort_faces(o, nb, *extra):
    order = np.lexsort((nb, o))
    return (o[order], nb[order]) + tuple(e[order] for e in extra)


def _one_norm(blocks):
    """Max column abs sum of each n x n block."""
    return np.abs(blocks).sum(axis=-2).max(axis=-1)


def _row_offdiag_sum(C, owner, neighbour, up_val, lo_val):
    # one pass over owner contributions then neighbour contributions, each
    # cell's sum accumulated in that order from 0.0
    idx = np.concatenate([owner, neighbour])
    return np.bincount(idx, weights=np.concatenate([up_val, lo_val]), minlength=C).astype(np.float64)


def _density_values(C, owner, neighbour, rng, n=5):
    F = owner.size
    G = rng.standard_normal((F, 2, n, n))
    eye = np.eye(n)
    upper = -eye + 0.1 * G[:, 0]
    lower = -eye + 0.1 * G[:, 1]
    del G
    Gc = rng.standard_normal((C, n, n))
    s = _row_offdiag_sum(C, owner, neighbour, _one_norm(upper), _one_norm(lower))
    diag = (1.05 * s)[:, None, None] * eye + 0.1 * Gc
    b = rng.uniform(-1.0, 1.0, (C, n))
    return diag, upper, lower, b


def _pack(C, owner, neighbour, diag, upper, lower, b, **meta):
    n = diag.shape[-1]
    d = dict(n_cells=int(C), n_faces=int(owner.size), n=int(n),
             owner=np.ascontiguousarray(owner, dtype=np.int32),
             neighbour=np.ascontiguousarray(neighbour, dtype=np.int32),
             diag=np.ascontiguousarray(diag, dtype=np.float64),
             upper=np.ascontiguousarray(upper, dtype=np.float64),
             lower=np.ascontiguousarray(lower, dtype=np.float64),
             b=np.ascontiguousarray(b, dtype=np.float64))
    d.update(meta)
    return d


def density(nx=16, ny=None, nz=None, seed=0):
    """Density-based coupled system (5x5 blocks: rho, rhoU, rhoE; Sec. 2.1).

    Off-diagonal blocks -I + 0.1 G, G ~ N(0,1); diagonal block
    (1.05 * sum of the row's off-diagonal block 1-norms) I + 0.1 G_c;
    b ~ U(-1, 1). The diagonal shift mimics the V/dtau term of the
    pseudo-time linearisation.
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    C = nx * ny * nz
    lo, hi, _ = _hex_faces(nx, ny, nz)
    owner, neighbour = _sort_faces(lo, hi)
    rng = np.random.default_rng(seed)
    diag, upper, lower, b = _density_values(C, owner, neighbour, rng)
    return _pack(C, owner, neighbour, diag, upper, lower, b,
                 name=f"density {nx}x{ny}x{nz} n=5 seed={seed}")


def pressure(nx=64, ny=None, nz=None, seed=1):
    """Pressure-based coupled system (4x4 blocks ordered p, Ux, Uy, Uz; Sec. 2.2).

    Cells are randomly renumbered. Per face f (area A_f ~ U(0.5, 1.5), area
    vector S_f along the grid axis pointing from owner to neighbour):
      uu: off-diagonal -A_f I3 + 0.05 Gu (both sides), diagonal
          1.05 * (sum of the row's off-diagonal uu 1-norms) I3 + 0.05 Gc;
      up (gradient, interpolation weight f_x = 1/2): owner row +0.5 S_f in
          upper and on its diagonal, neighbour row -0.5 S_f in lower and on
          its diagonal;
      pp: a_f = A_f D_f, D_f = (1/abar_o + 1/abar_n) / 2 with abar the mean
          of the cell's uu diagonal; off-diagonal +a_f, diagonal -sum a_f;
          cells on the x = max boundary add -2 / abar (outlet pin);
      pu (divergence): the continuity row is written with the same overall
          sign as its pp entries, i.e. the negated divergence: owner row
          -0.5 S_f in upper and on its diagonal, neighbour row +0.5 S_f.
    Sec. 2.2 prints pp with off-diagonal +a and diagonal -a (the continuity
    equation times -1) but pu with the divergence's own sign; taken literally
    the pressure Schur complement nearly cancels and the system is close to
    singular. The continuity row here is negated as a whole.
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    C = nx * ny * nz
    rng = np.random.default_rng(seed)
    perm = rng.permutation(C)
    lo, hi, axis = _hex_faces(nx, ny, nz)
    a, b_ = perm[lo], perm[hi]
    owner = np.minimum(a, b_)
    neighbour = np.maximum(a, b_)
    sign = np.where(a < b_, 1.0, -1.0)          # +1 when the owner is the geometric lower cell
    owner, neighbour, axis, sign = _sort_faces(owner, neighbour, axis, sign)
    F = owner.size
    Af = rng.uniform(0.5, 1.5, F)
    Gu = rng.standard_normal((F, 2, 3, 3))
    Gc = rng.standard_normal((C, 3, 3))
    rhs = rng.uniform(-1.0, 1.0, (C, 4))

    S = np.zeros((F, 3))
    S[np.arange(F), axis] = Af * sign
    eye3 = np.eye(3)
    upper = np.zeros((F, 4, 4))
    lower = np.zeros((F, 4, 4))
    diag = np.zeros((C, 4, 4))
    upper[:, 1:, 1:] = -Af[:, None, None] * eye3 + 0.05 * Gu[:, 0]
    lower[:, 1:, 1:] = -Af[:, None, None] * eye3 + 0.05 * Gu[:, 1]
    s = _row_offdiag_sum(C, owner, neighbour, _one_norm(upper[:, 1:, 1:]), _one_norm(lower[:, 1:, 1:]))
    diag[:, 1:, 1:] = (1.05 * s)[:, None, None] * eye3 + 0.05 * Gc
    # momentum rows, pressure column (gradient) and its transpose (divergence)
    upper[:, 1:, 0] = 0.5 * S
    lower[:, 1:, 0] = -0.5 * S
    upper[:, 0, 1:] = -0.5 * S
    lower[:, 0, 1:] = 0.5 * S
    np.add.at(diag[:, 1:, 0], owner, 0.5 * S)
    np.add.at(diag[:, 1:, 0], neighbour, -0.5 * S)
    np.add.at(diag[:, 0, 1:], owner, -0.5 * S)
    np.add.at(diag[:, 0, 1:], neighbour, 0.5 * S)
    # pressure Laplacian from the Rhie-Chow term
    abar = np.trace(diag[:, 1:, 1:], axis1=1, axis2=2) / 3.0
    Df = 0.5 * (1.0 / abar[owner] + 1.0 / abar[neighbour])
    af = Af * Df
    upper[:, 0, 0] = af
    lower[:, 0, 0] = af
    pp = np.zeros(C)
    np.add.at(pp, owner, -af)
    np.add.at(pp, neighbour, -af)
    # outlet pin on the x = max boundary (lattice i == nx - 1)
    lattice_outlet = np.arange(C).reshape(nz, ny, nx)[:, :, nx - 1].ravel()
    out_cells = perm[lattice_outlet]
    pp[out_cells] += -2.0 / abar[out_cells]
    diag[:, 0, 0] = pp
    return _pack(C, owner, neighbour, diag, upper, lower, rhs,
                 name=f"pressure {nx}x{ny}x{nz} n=4 seed={seed}")


def knn(side=160, seed=3, kmin=4, kmax=12):
    """Unstructured 5x5 system: side^3 jittered lattice points, faces to k-NN.

    Points are lattice points plus U(-0.3, 0.3) of the spacing per coordinate;
    each point i draws k_i ~ U{kmin..kmax} and links to its k_i nearest
    neighbours; the link set is symmetrised (union) and deduplicated. Values
    follow density().
    """
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    C = side ** 3
    g = np.arange(side, dtype=np.float64)
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)[:, ::-1].copy()
    pts += rng.uniform(-0.3, 0.3, pts.shape)
    k = rng.integers(kmin, kmax + 1, C)
    tree = cKDTree(pts)
    _, nbrs = tree.query(pts, k=kmax + 1, workers=-1)
    nbrs = nbrs[:, 1:]
    keep = np.arange(kmax)[None, :] < k[:, None]
    src = np.repeat(np.arange(C), kmax).reshape(C, kmax)[keep]
    dst = nbrs[keep]
    o = np.minimum(src, dst).astype(np.int64)
    nb = np.maximum(src, dst).astype(np.int64)
    key = np.sort(o * C + nb)
    key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    owner = (key // C).astype(np.int64)
    neighbour = (key % C).astype(np.int64)
    diag, upper, lower, b = _density_values(C, owner, neighbour, rng)
    return _pack(C, owner, neighbour, diag, upper, lower, b,
                 name=f"knn {side}^3 k={kmin}..{kmax} n=5 seed={seed}")


def random_graph(C, F, n, seed, dominance=1.05):
    """Small random LDU system on a random simple graph (test inputs)."""
    rng = np.random.default_rng(seed)
    pairs = set()
    while len(pairs) < F:
        i, j = rng.integers(0, C, 2)
        if i != j:
            pairs.add((int(min(i, j)), int(max(i, j))))
    pairs = sorted(pairs)
    owner = np.array([p[0] for p in pairs], dtype=np.int64)
    neighbour = np.array([p[1] for p in pairs], dtype=np.int64)
    G = rng.standard_normal((F, 2, n, n))
    eye = np.eye(n)
    upper = -eye + 0.3 * G[:, 0]
    lower = -eye + 0.3 * G[:, 1]
    s = _row_offdiag_sum(C, owner, neighbour, _one_norm(upper), _one_norm(lower))
    diag = (dominance * s + 1.0)[:, None, None] * eye + 0.3 * rng.standard_normal((C, n, n))
    b = rng.uniform(-1.0, 1.0, (C, n))
    return _pack(C, owner, neighbour, diag, upper, lower, b, name=f"random C={C} F={F} n={n}")


def perturb(sys, rng, eps=0.02):
    """Values-only update: every coefficient times 1 + eps * U(-1, 1)."""
    out = dict(sys)
    for key in ("diag", "upper", "lower"):
        a = sys[key]
        out[key] = np.ascontiguousarray(a * (1.0 + eps * rng.uniform(-1.0, 1.0, a.shape)))
    return out


CONFIGS = {
    "c1": lambda: density(16, seed=0),
    "c2": lambda: pressure(64, seed=1),
    "c3": lambda: density(128, seed=2),
    "c4": lambda: knn(160, seed=3),
}


def flow(nx=16, ny=None, nz=None, seed=5, gamma=1.4, mach=0.5, skew=False):
    """Flow state and face geometry for assembling the density-based system
    (Sec. 2.1) on an nx*ny*nz hex grid of cubic cells, spacing h = 1/nx.

    Per cell (x, y, z the cell centre), with N ~ N(0, 1) drawn in this order:
        rho = 1 + 0.1 sin(2 pi x) cos(2 pi y) + 0.02 N
        p   = (1 + 0.1 cos(2 pi z) + 0.02 N) / gamma        (sound speed ~ 1)
        u   = mach * (1 + 0.1 N, 0.2 sin(2 pi x) + 0.1 N, 0.1 N)
        Q   = (rho, rho u, rho v, rho w, p / (gamma - 1) + rho |u|^2 / 2)
    then b ~ U(-1, 1) per unknown. Faces as density() (owner < neighbour,
    upper-triangular order) with area h^2, unit normal along +axis (owner to
    neighbour) and centre distance h. skew=True then perturbs the geometry:
    normal = unit(axis + 0.3 N^3), area and distance x (1 + 0.2 U(-1, 1)).
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    C = nx * ny * nz
    h = 1.0 / nx
    lo, hi, axis = _hex_faces(nx, ny, nz)
    owner, neighbour, axis = _sort_faces(lo, hi, axis)
    F = owner.size
    idx = np.arange(C)
    x = (idx % nx + 0.5) * h
    y = ((idx // nx) % ny + 0.5) * h
    z = (idx // (nx * ny) + 0.5) * h
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.1 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) + 0.02 * rng.standard_normal(C)
    p = (1.0 + 0.1 * np.cos(2 * np.pi * z) + 0.02 * rng.standard_normal(C)) / gamma
    N = rng.standard_normal((C, 3))
    u = mach * np.stack([1.0 + 0.1 * N[:, 0], 0.2 * np.sin(2 * np.pi * x) + 0.1 * N[:, 1], 0.1 * N[:, 2]], -1)
    Q = np.empty((C, 5))
    Q[:, 0] = rho
    Q[:, 1:4] = rho[:, None] * u
    Q[:, 4] = p / (gamma - 1.0) + 0.5 * rho * (u * u).sum(-1)
    b = rng.uniform(-1.0, 1.0, (C, 5))
    normal = np.zeros((F, 3))
    normal[np.arange(F), axis] = 1.0
    area = np.full(F, h * h)
    dist = np.full(F, h)
    if skew:
        normal += 0.3 * rng.standard_normal((F, 3))
        normal /= np.linalg.norm(normal, axis=1, keepdims=True)
        area *= 1.0 + 0.2 * rng.uniform(-1.0, 1.0, F)
        dist *= 1.0 + 0.2 * rng.uniform(-1.0, 1.0, F)
    return dict(n_cells=int(C), n_faces=int(F), n=5,
                owner=np.ascontiguousarray(owner, dtype=np.int32),
                neighbour=np.ascontiguousarray(neighbour, dtype=np.int32),
                Q=np.ascontiguousarray(Q), area=np.ascontiguousarray(area),
                normal=np.ascontiguousarray(normal), dist=np.ascontiguousarray(dist),
                b=np.ascontiguousarray(b), gamma=gamma,
                name=f"flow {nx}x{ny}x{nz} mach={mach} seed={seed}{' skewed' if skew else ''}")
