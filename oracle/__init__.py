"""ctypes wrapper of the FP64 CPU oracle (oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by the tests, the package smoke check and
the benchmark's CPU-baseline leg. The product path never imports this module.
"""
import ctypes as ct
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.cpp")
_SRCS = [_SRC, os.path.join(_HERE, "assembly.cpp"), os.path.join(_HERE, "reorder.cpp")]

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


class Config(ct.Structure):
    _fields_ = [
        ("solver", ct.c_int), ("restart", ct.c_int), ("tol", ct.c_double),
        ("maxiter", ct.c_int), ("precond", ct.c_int), ("pmode", ct.c_int),
        ("matching_rounds", ct.c_int), ("agg_passes", ct.c_int),
        ("jacobi_omega", ct.c_double), ("nu1", ct.c_int), ("nu2", ct.c_int),
        ("coarse_size", ct.c_int), ("max_levels", ct.c_int),
        ("max_coarsen_ratio", ct.c_double), ("p_omega", ct.c_double),
        ("coarse_dense_max", ct.c_int), ("coarse_sweeps", ct.c_int), ("smoother", ct.c_int),
    ]


class Result(ct.Structure):
    _fields_ = [("status", ct.c_int), ("iters", ct.c_int), ("restarts", ct.c_int),
                ("rel_res_initial", ct.c_double), ("rel_res_final", ct.c_double),
                ("levels", ct.c_int)]


_SO_OMP = os.path.join(_HERE, "liboracle_omp.so")


def build(force=False, omp=False):
    """Compile liboracle.so (plain C++17, no implicit FMA contraction,
    single-threaded), or with omp=True liboracle_omp.so: the same source
    with its OpenMP pragmas enabled. Those sit only on loops whose
    iterations write disjoint outputs (the row loops of the SpMV and the
    sweeps, element-wise vector updates); no reduction is split, so both
    builds give identical results."""
    so = _SO_OMP if omp else _SO
    if not force and os.path.exists(so) and os.path.getmtime(so) >= max(
            [os.path.getmtime(p) for p in _SRCS] + [os.path.getmtime(os.path.join(_HERE, "oracle.h"))]):
        return so
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared"] + (["-fopenmp"] if omp else []) + ["-o", so] + _SRCS
    subprocess.check_call(cmd)
    return so


_lib = None
_omp = False


def use_openmp(flag=True):
    """Switch this process to the OpenMP build (all host cores) or back to
    the single-threaded one; takes effect at the next call."""
    global _lib, _omp
    if bool(flag) != _omp:
        _omp = bool(flag)
        _lib = None


def lib():
    global _lib
    if _lib is None:
        so = build(omp=_omp)
        L = ct.CDLL(so)
        L.or_config_default.argtypes = [ct.POINTER(Config)]
        L.or_ldu_check.argtypes = [ct.c_int, ct.c_int, _i32p, _i32p]
        L.or_ldu_structure.argtypes = [ct.c_int, ct.c_int, _i32p, _i32p, _i32p, _i32p, _i32p, _i32p, _i32p]
        L.or_ldu_values.argtypes = [ct.c_int, ct.c_int, ct.c_int, _i32p, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p]
        L.or_bsr_to_ldu.argtypes = [ct.c_int, ct.c_int, ct.c_int, _i32p, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p]
        L.or_bsr_spmv.argtypes = [ct.c_int, ct.c_int, _i32p, _i32p, _f64p, _f64p, _f64p]
        L.or_dense_inverse.argtypes = [ct.c_int, _f64p, _f64p]
        L.or_block_norms.argtypes = [ct.c_int, ct.c_int, _f64p, _f64p]
        L.or_aggregate.argtypes = [ct.c_int, ct.c_int, _i32p, _i32p, _f64p, ct.POINTER(Config), _i32p]
        L.or_amg_setup.restype = ct.c_void_p
        L.or_amg_setup.argtypes = [ct.c_int, ct.c_int, _i32p, _i32p, _f64p, ct.POINTER(Config), ct.POINTER(ct.c_int)]
        L.or_amg_resetup.argtypes = [ct.c_void_p, _f64p]
        L.or_amg_free.argtypes = [ct.c_void_p]
        L.or_amg_levels.argtypes = [ct.c_void_p]
        L.or_amg_level_info.argtypes = [ct.c_void_p, ct.c_int] + [ct.POINTER(ct.c_int)] * 4
        L.or_amg_get_A.argtypes = [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p]
        L.or_amg_get_P.argtypes = [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]
        L.or_amg_get_dinv.argtypes = [ct.c_void_p, ct.c_int, _f64p]
        L.or_amg_get_coarse_inverse.argtypes = [ct.c_void_p, _f64p]
        L.or_amg_vcycle.argtypes = [ct.c_void_p, _f64p, _f64p]
        L.or_amg_get_dilu.argtypes = [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p]
        L.or_colour.argtypes = [ct.c_int, _i32p, _i32p, _i32p]
        L.or_dilu_factor.argtypes = [ct.c_int, ct.c_int, _i32p, _i32p, _f64p, _i32p, _f64p]
        L.or_dilu_apply.argtypes = [ct.c_int, ct.c_int, _i32p, _i32p, _f64p, _i32p, ct.c_int, _f64p, _f64p, _f64p]
        L.or_solve.argtypes = [ct.c_int, ct.c_int, _i32p, _i32p, _f64p, ct.c_void_p, ct.POINTER(Config),
                               _f64p, _f64p, ct.POINTER(Result), ct.c_void_p, ct.c_int]
        L.or_solve_trace.argtypes = [ct.c_int, ct.c_int, _i32p, _i32p, _f64p, ct.c_void_p, ct.POINTER(Config),
                                     _f64p, _f64p, ct.POINTER(Result), ct.c_void_p, ct.c_int,
                                     ct.c_void_p, ct.c_void_p, ct.c_int]
        L.or_fgmres_arnoldi.argtypes = [ct.c_int, ct.c_int, _i32p, _i32p, _f64p, ct.c_void_p,
                                        ct.POINTER(Config), _f64p, ct.c_int, _f64p, _f64p, _f64p]
        L.or_rcm.argtypes = [ct.c_int, ct.c_int, _i32p, _i32p, _i32p]
        d3 = [_f64p, _f64p, ct.c_double, _f64p]
        L.or_euler_flux.argtypes = d3
        L.or_flux_jacobian.argtypes = d3
        L.or_face_lambda.argtypes = [_f64p, _f64p, _f64p, ct.c_double, ct.c_double, ct.c_double, ct.c_double,
                                     ct.POINTER(ct.c_double)]
        L.or_assemble_density.argtypes = [ct.c_int, ct.c_int, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p,
                                          ct.c_double, ct.c_double, ct.c_double, ct.c_double, _f64p, _f64p, _f64p]
        _lib = L
    return _lib


def config(**kw):
    c = Config()
    lib().or_config_default(ct.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


def _p(a):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def ldu_check(C, owner, neighbour):
    owner = np.ascontiguousarray(owner, np.int32)
    neighbour = np.ascontiguousarray(neighbour, np.int32)
    return lib().or_ldu_check(C, owner.size, owner, neighbour)


def ldu_to_bsr(sys):
    """Block-CSR structure and values of an LDU system (dict from synth)."""
    C, F, n = sys["n_cells"], sys["n_faces"], sys["n"]
    owner = np.ascontiguousarray(sys["owner"], np.int32)
    nb = np.ascontiguousarray(sys["neighbour"], np.int32)
    rp = np.zeros(C + 1, np.int32)
    col = np.zeros(C + 2 * F, np.int32)
    pd = np.zeros(C, np.int32)
    pu = np.zeros(F, np.int32)
    pl = np.zeros(F, np.int32)
    st = lib().or_ldu_structure(C, F, owner, nb, rp, col, pd, pu, pl)
    if st:
        raise ValueError("invalid LDU addressing")
    val = np.zeros((C + 2 * F) * n * n)
    lib().or_ldu_values(C, F, n, pd, pu, pl, sys["diag"].ravel(), sys["upper"].ravel(),
                        sys["lower"].ravel(), val)
    return dict(rows=C, n=n, row_ptr=rp, col=col, val=val.reshape(-1, n, n),
                pos_diag=pd, pos_up=pu, pos_lo=pl)


def bsr_to_ldu(bsr, F):
    C, n = bsr["rows"], bsr["n"]
    d = np.zeros(C * n * n)
    u = np.zeros(F * n * n)
    lo = np.zeros(F * n * n)
    lib().or_bsr_to_ldu(C, F, n, bsr["pos_diag"], bsr["pos_up"], bsr["pos_lo"],
                        np.ascontiguousarray(bsr["val"]).ravel(), d, u, lo)
    return d.reshape(C, n, n), u.reshape(F, n, n), lo.reshape(F, n, n)


def spmv(bsr, x):
    rows, n = bsr["rows"], bsr["n"]
    y = np.zeros(rows * n)
    lib().or_bsr_spmv(rows, n, bsr["row_ptr"], bsr["col"], np.ascontiguousarray(bsr["val"]).ravel(),
                      np.ascontiguousarray(x, np.float64).ravel(), y)
    return y.reshape(rows, n)


def dense_inverse(A):
    A = np.ascontiguousarray(A, np.float64)
    N = A.shape[0]
    out = np.zeros((N, N))
    if lib().or_dense_inverse(N, A.ravel(), out.ravel()):
        raise np.linalg.LinAlgError("zero pivot")
    return out


def block_norms(val):
    val = np.ascontiguousarray(val, np.float64)
    nb, n = val.shape[0], val.shape[1]
    out = np.zeros(nb)
    lib().or_block_norms(nb, n, val.ravel(), out)
    return out


def aggregate(bsr, cfg=None):
    cfg = cfg or config()
    agg = np.zeros(bsr["rows"], np.int32)
    na = lib().or_aggregate(bsr["rows"], bsr["n"], bsr["row_ptr"], bsr["col"],
                            np.ascontiguousarray(bsr["val"]).ravel(), ct.byref(cfg), agg)
    return agg, na


class Amg:
    """AMG hierarchy built by the oracle (full setup at construction)."""

    def __init__(self, bsr, cfg=None):
        self.cfg = cfg or config()
        self.n = bsr["n"]
        self.rows = bsr["rows"]
        self._bsr = bsr
        st = ct.c_int(0)
        self.h = lib().or_amg_setup(bsr["rows"], bsr["n"], bsr["row_ptr"], bsr["col"],
                                    np.ascontiguousarray(bsr["val"]).ravel(), ct.byref(self.cfg), ct.byref(st))
        self.status = st.value

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_amg_free(self.h)
            self.h = None

    def resetup(self, val):
        return lib().or_amg_resetup(self.h, np.ascontiguousarray(val, np.float64).ravel())

    @property
    def levels(self):
        return lib().or_amg_levels(self.h)

    def info(self, l):
        r, nz, pn, k = ct.c_int(), ct.c_int(), ct.c_int(), ct.c_int()
        lib().or_amg_level_info(self.h, l, ct.byref(r), ct.byref(nz), ct.byref(pn), ct.byref(k))
        return dict(rows=r.value, nnz=nz.value, p_nnz=pn.value, coarse_kind=k.value)

    def A(self, l):
        i = self.info(l)
        n = self.n
        rp = np.zeros(i["rows"] + 1, np.int32)
        ci = np.zeros(i["nnz"], np.int32)
        v = np.zeros(i["nnz"] * n * n)
        lib().or_amg_get_A(self.h, l, _p(rp), _p(ci), _p(v))
        return dict(rows=i["rows"], n=n, row_ptr=rp, col=ci, val=v.reshape(-1, n, n))

    def P(self, l):
        i = self.info(l)
        n = self.n
        rp = np.zeros(i["rows"] + 1, np.int32)
        ci = np.zeros(i["p_nnz"], np.int32)
        v = np.zeros(i["p_nnz"] * n * n)
        agg = np.zeros(i["rows"], np.int32)
        om = ct.c_double(0)
        lib().or_amg_get_P(self.h, l, _p(rp), _p(ci), _p(v), _p(agg), ct.byref(om))
        cols = self.info(l + 1)["rows"]
        return dict(rows=i["rows"], cols=cols, n=n, row_ptr=rp, col=ci, val=v.reshape(-1, n, n),
                    agg=agg, omega=om.value)

    def dinv(self, l):
        i = self.info(l)
        out = np.zeros(i["rows"] * self.n * self.n)
        lib().or_amg_get_dinv(self.h, l, out)
        return out.reshape(-1, self.n, self.n)

    def coarse_inverse(self):
        i = self.info(self.levels - 1)
        N = i["rows"] * self.n
        out = np.zeros(N * N)
        lib().or_amg_get_coarse_inverse(self.h, out)
        return out.reshape(N, N)

    def dilu(self, l):
        """(number of colours, colour[rows], einv[rows][n][n]) of level l, or
        (-1, None, None) when the level keeps block Jacobi."""
        rows = self.info(l)["rows"]
        n = self.n
        col = np.zeros(rows, np.int32)
        einv = np.zeros((rows, n, n))
        nc = lib().or_amg_get_dilu(self.h, l, _p(col), _p(einv))
        return (nc, col, einv) if nc > 0 else (-1, None, None)

    def vcycle(self, v):
        v = np.ascontiguousarray(v, np.float64).ravel()
        z = np.zeros_like(v)
        lib().or_amg_vcycle(self.h, v, z)
        return z.reshape(-1, self.n)


def solve(bsr, b, x0=None, cfg=None, amg=None, hist_len=0):
    """Krylov solve with the oracle; returns (x, result dict, history)."""
    cfg = cfg or config()
    n, rows = bsr["n"], bsr["rows"]
    if cfg.precond == 0 and amg is None:
        amg = Amg(bsr, cfg)
        if amg.status:
            return None, dict(status=amg.status), None
    x = np.zeros(rows * n) if x0 is None else np.ascontiguousarray(x0, np.float64).ravel().copy()
    res = Result()
    hist = np.zeros(max(hist_len, 1))
    lib().or_solve(rows, n, bsr["row_ptr"], bsr["col"], np.ascontiguousarray(bsr["val"]).ravel(),
                   amg.h if amg is not None else None, ct.byref(cfg),
                   np.ascontiguousarray(b, np.float64).ravel(), x, ct.byref(res),
                   _p(hist) if hist_len else None, hist_len)
    out = {k: getattr(res, k) for k, _ in Result._fields_}
    return x.reshape(rows, n), out, hist[:min(hist_len, res.iters)] if hist_len else None


def bicgstab_trace(bsr, b, cfg, amg=None, max_iters=200):
    """BiCGStab (cfg.solver must be 1) with its per-iteration iterates x_k
    and recurrence residuals: (x, result dict, xs[k], rs[k])."""
    assert cfg.solver == 1
    n, rows = bsr["n"], bsr["rows"]
    N = rows * n
    x = np.zeros(N)
    res = Result()
    xs = np.zeros((max_iters, N))
    rs = np.zeros((max_iters, N))
    cnt = lib().or_solve_trace(rows, n, bsr["row_ptr"], bsr["col"], np.ascontiguousarray(bsr["val"]).ravel(),
                               amg.h if amg is not None else None, ct.byref(cfg),
                               np.ascontiguousarray(b, np.float64).ravel(), x, ct.byref(res), None, 0,
                               _p(xs), _p(rs), max_iters)
    out = {k: getattr(res, k) for k, _ in Result._fields_}
    return x.reshape(rows, n), out, xs[:cnt], rs[:cnt]


def arnoldi(bsr, b, j_steps, cfg=None, amg=None):
    cfg = cfg or config()
    n, rows = bsr["n"], bsr["rows"]
    N = rows * n
    V = np.zeros((j_steps + 1) * N)
    Z = np.zeros(j_steps * N)
    H = np.zeros((j_steps + 1) * j_steps)
    done = lib().or_fgmres_arnoldi(rows, n, bsr["row_ptr"], bsr["col"], np.ascontiguousarray(bsr["val"]).ravel(),
                                   amg.h if amg is not None else None, ct.byref(cfg),
                                   np.ascontiguousarray(b, np.float64).ravel(), j_steps, V, Z, H)
    return done, V.reshape(j_steps + 1, N), Z.reshape(j_steps, N), H.reshape(j_steps + 1, j_steps)


def colour(bsr):
    """Multicolouring of a BSR pattern: (number of colours or -1, colour[rows])."""
    col = np.zeros(bsr["rows"], np.int32)
    nc = lib().or_colour(bsr["rows"], bsr["row_ptr"], bsr["col"], col)
    return nc, col


def dilu_factor(bsr, colour_):
    """DILU block inverses E_i^{-1} for a colouring: (status, einv)."""
    n = bsr["n"]
    einv = np.zeros((bsr["rows"], n, n))
    st = lib().or_dilu_factor(bsr["rows"], n, bsr["row_ptr"], bsr["col"],
                              np.ascontiguousarray(bsr["val"], np.float64).ravel(),
                              np.ascontiguousarray(colour_, np.int32), einv.reshape(-1))
    return st, einv


def dilu_apply(bsr, colour_, einv, r):
    """z = M^{-1} r for the DILU factorisation (einv) of bsr."""
    n = bsr["n"]
    z = np.zeros((bsr["rows"], n))
    lib().or_dilu_apply(bsr["rows"], n, bsr["row_ptr"], bsr["col"],
                        np.ascontiguousarray(bsr["val"], np.float64).ravel(),
                        np.ascontiguousarray(colour_, np.int32), int(np.max(colour_)) + 1,
                        np.ascontiguousarray(einv, np.float64).ravel(),
                        np.ascontiguousarray(r, np.float64).ravel(), z.reshape(-1))
    return z


# ---- assembly of the density-based system (assembly.cpp) -------------------
FLOW_DEFAULTS = dict(gamma=1.4, mu=1e-3, prandtl=0.72, cfl=10.0)


def _f64(a):
    return np.ascontiguousarray(a, np.float64)


def euler_flux(Q, n, gamma=1.4):
    """Inviscid normal flux F(Q, n) of one state; None for an invalid state."""
    F = np.zeros(5)
    return None if lib().or_euler_flux(_f64(Q), _f64(n), gamma, F) else F


def flux_jacobian(Q, n, gamma=1.4):
    """J(Q, n) = dF/dQ (5 x 5); None for an invalid state."""
    J = np.zeros(25)
    return None if lib().or_flux_jacobian(_f64(Q), _f64(n), gamma, J) else J.reshape(5, 5)


def face_lambda(Qo, Qn, n, d, gamma=1.4, mu=1e-3, prandtl=0.72):
    lam = ct.c_double()
    st = lib().or_face_lambda(_f64(Qo), _f64(Qn), _f64(n), d, gamma, mu, prandtl, ct.byref(lam))
    return None if st else lam.value


def assemble_density(flow, **prm):
    """LDU blocks (diag, upper, lower) of the density-based system from a
    flow dict (synth.flow); (status, diag, upper, lower)."""
    p = dict(FLOW_DEFAULTS, **prm)
    C, F = flow["n_cells"], flow["n_faces"]
    diag = np.zeros((C, 5, 5))
    upper = np.zeros((F, 5, 5))
    lower = np.zeros((F, 5, 5))
    st = lib().or_assemble_density(C, F, flow["owner"], flow["neighbour"], _f64(flow["Q"]).ravel(),
                                   _f64(flow["area"]), _f64(flow["normal"]).ravel(), _f64(flow["dist"]),
                                   p["gamma"], p["mu"], p["prandtl"], p["cfl"], diag.reshape(-1),
                                   upper.reshape(-1), lower.reshape(-1))
    return st, diag, upper, lower


# ---- segregated fields <-> block AoS (Alg. 1 steps 1, 5 and 15) -------------
# A coupled system's unknowns come as a list of fields, field k with ncomp[k]
# components per cell (1: scalar field, 3: vector field stored [cell][3]); the
# block unknown order is the fields' order with each field's components in
# turn. Plain definitions with numpy.

def field_offsets(ncomp):
    return np.concatenate(([0], np.cumsum(ncomp))).astype(int)


def pack_vector(fields, ncomp):
    """Block AoS vector [C][n] from the list of fields (Alg. 1 step 1)."""
    C = fields[0].size // ncomp[0]
    off = field_offsets(ncomp)
    out = np.zeros((C, off[-1]))
    for k, f in enumerate(fields):
        out[:, off[k]:off[k + 1]] = np.asarray(f, np.float64).reshape(C, ncomp[k])
    return out


def unpack_vector(vec, ncomp):
    """The list of fields from a block AoS vector (Alg. 1 step 15)."""
    off = field_offsets(ncomp)
    vec = np.asarray(vec).reshape(vec.shape[0], off[-1])
    return [np.ascontiguousarray(vec[:, off[k]:off[k + 1]]).reshape(-1) for k in range(len(ncomp))]


def pack_coefficients(coupling, ncomp, C, F):
    """LDU blocks diag[C][n][n], upper / lower[F][n][n] (Alg. 1 step 5) from
    the couplings: coupling[a][b] = (diag, upper, lower) with ncomp[a] x
    ncomp[b] row-major sub-blocks, or None for a zero coupling."""
    off = field_offsets(ncomp)
    n = off[-1]
    out = [np.zeros((C, n, n)), np.zeros((F, n, n)), np.zeros((F, n, n))]
    for a in range(len(ncomp)):
        for b in range(len(ncomp)):
            cp = coupling[a][b]
            if cp is None:
                continue
            for o, src, m in zip(out, cp, (C, F, F)):
                o[:, off[a]:off[a + 1], off[b]:off[b + 1]] = np.asarray(src, np.float64).reshape(m, ncomp[a], ncomp[b])
    return out


# ---- locality ordering (reorder.cpp) ----------------------------------------
def rcm(C, owner, neighbour):
    """Reverse Cuthill-McKee permutation perm[new] = old; None for bad faces."""
    perm = np.zeros(C, np.int32)
    st = lib().or_rcm(C, len(owner), np.ascontiguousarray(owner, np.int32),
                      np.ascontiguousarray(neighbour, np.int32), perm)
    return None if st else perm
