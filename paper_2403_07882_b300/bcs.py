"""Python binding of the C ABI in include/bcs.h (argument marshalling only).

Every function named bcs_* here calls the library function of the same name.
Arrays may be numpy arrays (host memory, BCS_MEM_HOST) or CUDA torch tensors
(device memory, BCS_MEM_DEVICE); all arrays of one call must live in the same
place. There is no fallback: without the built CUDA library (libbcs.so) every
call raises.
"""
import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbcs.so")

BCS_OK, BCS_EINVAL, BCS_ENOMEM, BCS_ECUDA, BCS_NOT_CONVERGED, BCS_BREAKDOWN, \
    BCS_SINGULAR_BLOCK, BCS_TIMEOUT, BCS_REJECTED, BCS_ESTATE = range(10)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "NOT_CONVERGED", "BREAKDOWN",
                "SINGULAR_BLOCK", "TIMEOUT", "REJECTED", "ESTATE"]
BCS_MEM_HOST, BCS_MEM_DEVICE = 0, 1
BCS_FGMRES, BCS_BICGSTAB = 0, 1
BCS_PC_AMG, BCS_PC_NONE, BCS_PC_JACOBI, BCS_PC_SGS = 0, 1, 2, 3
BCS_P_SMOOTHED, BCS_P_TENTATIVE = 0, 1
BCS_PREC_FP64, BCS_PREC_FP32, BCS_PREC_BF16 = 0, 1, 2
BCS_SMOOTH_JACOBI, BCS_SMOOTH_DILU, BCS_SMOOTH_SGS = 0, 1, 2
NUM_KERNEL_KINDS = 16


# device allocator callbacks of bcs_config
ALLOC_FN = ct.CFUNCTYPE(ct.c_void_p, ct.c_size_t, ct.c_void_p, ct.c_void_p)
RELEASE_FN = ct.CFUNCTYPE(None, ct.c_void_p, ct.c_size_t, ct.c_void_p, ct.c_void_p)


class bcs_config(ct.Structure):
    _fields_ = [
        ("solver", ct.c_int), ("restart", ct.c_int), ("tol", ct.c_double), ("maxiter", ct.c_int),
        ("precond", ct.c_int), ("pmode", ct.c_int), ("matching_rounds", ct.c_int),
        ("agg_passes", ct.c_int), ("jacobi_omega", ct.c_double), ("nu1", ct.c_int), ("nu2", ct.c_int),
        ("coarse_size", ct.c_int), ("max_levels", ct.c_int), ("max_coarsen_ratio", ct.c_double),
        ("p_omega", ct.c_double), ("coarse_dense_max", ct.c_int), ("coarse_sweeps", ct.c_int),
        ("precision", ct.c_int), ("smoother", ct.c_int), ("profile", ct.c_int), ("profile_kinds", ct.c_int),
        ("slice_layout", ct.c_int), ("cycle_graph", ct.c_int), ("reorder", ct.c_int), ("tail_rows", ct.c_int),
        ("dilu_cluster_rows", ct.c_int), ("dependent_launch", ct.c_int), ("x0_zero", ct.c_int),
        ("alloc", ALLOC_FN), ("release", RELEASE_FN), ("alloc_user", ct.c_void_p),
    ]


class bcs_result(ct.Structure):
    _fields_ = [("status", ct.c_int), ("iters", ct.c_int), ("restarts", ct.c_int), ("levels", ct.c_int),
                ("rel_res_initial", ct.c_double), ("rel_res_final", ct.c_double),
                ("setup_ms", ct.c_double), ("solve_ms", ct.c_double), ("host_syncs", ct.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class bcs_stats(ct.Structure):
    _fields_ = [("launches", ct.c_longlong), ("kind_launches", ct.c_longlong * NUM_KERNEL_KINDS),
                ("kind_ms", ct.c_double * NUM_KERNEL_KINDS), ("kind_bytes", ct.c_double * NUM_KERNEL_KINDS),
                ("kind_flops", ct.c_double * NUM_KERNEL_KINDS)]


class bcs_server_stats(ct.Structure):
    _fields_ = [("submitted", ct.c_longlong), ("completed", ct.c_longlong), ("rejected", ct.c_longlong),
                ("evictions", ct.c_longlong), ("admissions", ct.c_longlong), ("queued", ct.c_longlong),
                ("resident_bytes", ct.c_size_t), ("budget_bytes", ct.c_size_t), ("resident_cases", ct.c_int),
                ("p50_ms", ct.c_double), ("p99_ms", ct.c_double), ("mean_ms", ct.c_double),
                ("window_ms", ct.c_double), ("busy_frac", ct.c_double), ("overlap_frac", ct.c_double),
                ("mean_in_flight", ct.c_double), ("batches", ct.c_longlong), ("batched_requests", ct.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class bcs_flow_params(ct.Structure):
    _fields_ = [("gamma", ct.c_double), ("mu", ct.c_double), ("prandtl", ct.c_double), ("cfl", ct.c_double)]


class bcs_coupling(ct.Structure):
    _fields_ = [("diag", ct.c_void_p), ("upper", ct.c_void_p), ("lower", ct.c_void_p)]


class BcsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 10 else status}: {msg}")
        self.status = status


_lib = None
_vp = ct.c_void_p


def lib():
    """The loaded CUDA library; raises when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run __graft_entry__.build() or python -m paper_2403_07882_b300.build)")
        L = ct.CDLL(LIB_PATH)
        sig = {
            "bcs_config_default": (ct.c_int, [ct.POINTER(bcs_config)]),
            "bcs_create": (ct.c_int, [ct.POINTER(_vp), ct.c_int, ct.POINTER(bcs_config), _vp]),
            "bcs_destroy": (ct.c_int, [_vp]),
            "bcs_set_config": (ct.c_int, [_vp, ct.POINTER(bcs_config)]),
            "bcs_set_structure": (ct.c_int, [_vp, ct.c_int32, ct.c_int32, _vp, _vp, ct.c_int]),
            "bcs_set_values": (ct.c_int, [_vp, _vp, _vp, _vp, ct.c_int]),
            "bcs_invalidate_hierarchy": (ct.c_int, [_vp]),
            "bcs_flow_params_default": (ct.c_int, [ct.POINTER(bcs_flow_params)]),
            "bcs_pack_vector": (ct.c_int, [_vp, ct.c_int, _vp, _vp, _vp, ct.c_int]),
            "bcs_get_permutation": (ct.c_int, [_vp, _vp]),
            "bcs_unpack_vector": (ct.c_int, [_vp, ct.c_int, _vp, _vp, _vp, ct.c_int]),
            "bcs_pack_coefficients": (ct.c_int, [_vp, ct.c_int, _vp, _vp, _vp, _vp, _vp, ct.c_int]),
            "bcs_assemble_density": (ct.c_int, [_vp] + [_vp] * 4 + [ct.POINTER(bcs_flow_params)] + [_vp] * 3
                                     + [ct.c_int]),
            "bcs_solve": (ct.c_int, [_vp, _vp, _vp, ct.c_int, ct.POINTER(bcs_result)]),
            "bcs_solve_batch": (ct.c_int, [ct.POINTER(_vp), ct.c_int, ct.POINTER(_vp), ct.POINTER(_vp), ct.c_int,
                                           ct.POINTER(bcs_result)]),
            "bcs_spmv": (ct.c_int, [_vp, _vp, _vp, ct.c_int]),
            "bcs_precond_apply": (ct.c_int, [_vp, _vp, _vp, ct.c_int]),
            "bcs_get_bsr": (ct.c_int, [_vp] + [_vp] * 6),
            "bcs_num_levels": (ct.c_int, [_vp]),
            "bcs_get_level_info": (ct.c_int, [_vp, ct.c_int] + [ct.POINTER(ct.c_int)] * 4),
            "bcs_get_level": (ct.c_int, [_vp, ct.c_int] + [_vp] * 5),
            "bcs_get_prolongation": (ct.c_int, [_vp, ct.c_int] + [_vp] * 3 + [ct.POINTER(ct.c_double)]),
            "bcs_get_coarse_inverse": (ct.c_int, [_vp, _vp]),
            "bcs_get_dilu": (ct.c_int, [_vp, ct.c_int, ct.POINTER(ct.c_int), _vp, _vp]),
            "bcs_get_stats": (ct.c_int, [_vp, ct.POINTER(bcs_stats)]),
            "bcs_reset_stats": (ct.c_int, [_vp]),
            "bcs_get_kernel_times": (ct.c_int, [_vp, ct.c_char_p, ct.c_size_t]),
            "bcs_kernel_kind_name": (ct.c_char_p, [ct.c_int]),
            "bcs_get_level_times": (ct.c_int, [_vp, ct.c_int, _vp, _vp, _vp]),
            "bcs_last_error": (ct.c_char_p, [_vp]),
            "bcs_device_bytes": (ct.c_size_t, [_vp]),
            "bcs_ldu_structure_noalloc": (ct.c_int, [ct.c_int32, ct.c_int32] + [_vp] * 8 + [ct.c_char_p, ct.c_size_t]),
            "bcs_server_create": (ct.c_int, [ct.POINTER(_vp), ct.c_size_t, ct.c_int, ct.POINTER(bcs_config)]),
            "bcs_server_destroy": (ct.c_int, [_vp]),
            "bcs_server_register_case": (ct.c_int, [_vp, ct.c_int, ct.c_int32, ct.c_int32, _vp, _vp,
                                                    ct.POINTER(ct.c_int)]),
            "bcs_server_submit": (ct.c_int, [_vp, ct.c_int, _vp, _vp, _vp, _vp, _vp, ct.c_int,
                                             ct.POINTER(ct.c_int64)]),
            "bcs_server_wait": (ct.c_int, [_vp, ct.c_int64, ct.c_int, ct.POINTER(bcs_result),
                                           ct.POINTER(ct.c_double)]),
            "bcs_server_get_stats": (ct.c_int, [_vp, ct.POINTER(bcs_server_stats)]),
            "bcs_server_set_batch": (ct.c_int, [_vp, ct.c_int]),
            "bcs_server_reset_stats": (ct.c_int, [_vp]),
            "bcs_server_last_error": (ct.c_int, [_vp, ct.c_char_p, ct.c_size_t]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_names():
    return ["bcs_config_default", "bcs_create", "bcs_destroy", "bcs_set_config", "bcs_set_structure",
            "bcs_set_values", "bcs_invalidate_hierarchy", "bcs_flow_params_default", "bcs_assemble_density",
            "bcs_pack_vector", "bcs_unpack_vector", "bcs_pack_coefficients", "bcs_get_permutation",
            "bcs_solve", "bcs_solve_batch", "bcs_spmv", "bcs_precond_apply",
            "bcs_get_bsr", "bcs_num_levels", "bcs_get_level_info", "bcs_get_level", "bcs_get_prolongation",
            "bcs_get_coarse_inverse", "bcs_get_dilu", "bcs_get_stats", "bcs_reset_stats", "bcs_get_kernel_times", "bcs_kernel_kind_name",
            "bcs_get_level_times", "bcs_last_error", "bcs_device_bytes", "bcs_ldu_structure_noalloc", "bcs_server_create",
            "bcs_server_destroy", "bcs_server_register_case", "bcs_server_submit", "bcs_server_wait",
            "bcs_server_get_stats", "bcs_server_reset_stats", "bcs_server_set_batch",
            "bcs_server_last_error"]


# ------------------------------------------------------------ marshalling
# Sizes the library cannot check (it receives bare pointers): per solver
# handle [n, C, F], per (server, case id) the case's [n, C, F].
_dims = {}


def _key(h):
    return h.value if isinstance(h, ct.c_void_p) else h


def _current_device():
    import torch
    return torch.cuda.current_device()


def _marshal(*specs):
    """Pointers and the memory kind of one call's arrays, validated first.

    specs: (array or None, dtype name, element count or None). Arrays are
    numpy arrays (host) or torch tensors (CUDA: device memory; CPU: host).
    Raises ValueError, before anything reaches the library, for a wrong
    dtype or element count, a non-contiguous array, a mix of host and
    device arrays, or a CUDA tensor on another device than the current one
    (the library launches on the current device)."""
    mems = set()
    ptrs = []
    for a, dt, count in specs:
        if a is None:
            ptrs.append(None)
            continue
        if isinstance(a, np.ndarray):
            if a.dtype != np.dtype(dt):
                raise ValueError(f"expected a {dt} array, got {a.dtype}")
            if not a.flags["C_CONTIGUOUS"]:
                raise ValueError("arrays must be C-contiguous")
            numel = a.size
            ptrs.append(a.ctypes.data)
            mems.add(BCS_MEM_HOST)
        else:  # torch tensor
            if str(a.dtype) != "torch." + dt:
                raise ValueError(f"expected a {dt} tensor, got {a.dtype}")
            if not a.is_contiguous():
                raise ValueError("tensors must be contiguous")
            numel = a.numel()
            if a.is_cuda:
                if a.device.index != _current_device():
                    raise ValueError(f"tensor on {a.device}, but the current CUDA device is "
                                     f"cuda:{_current_device()}")
                mems.add(BCS_MEM_DEVICE)
            else:
                mems.add(BCS_MEM_HOST)
            ptrs.append(a.data_ptr())
        if count is not None and numel != count:
            raise ValueError(f"expected {count} elements, got {numel}")
    if len(mems) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return ptrs, (mems.pop() if mems else BCS_MEM_HOST)


def _solver_dims(h):
    """(n, C, F) of a solver handle; C and F are None before set_structure
    (the library then refuses the call with BCS_ESTATE, touching no array)."""
    d = _dims.get(_key(h))
    if d is None:
        raise ValueError("unknown or destroyed solver handle")
    return d[0], (d[1] if d[1] > 0 else None), (d[2] if d[1] > 0 else None)


def _cnt(*factors):
    """Product of the factors; None (no size check: the library judges the
    call) when one is unknown or not positive."""
    out = 1
    for f in factors:
        if f is None or f <= 0:
            return None
        out *= f
    return out


def _check(status, handle=None):
    if status != BCS_OK:
        msg = lib().bcs_last_error(handle).decode() if handle else ""
        raise BcsError(status, msg)
    return status


def bcs_config_default(**overrides):
    c = bcs_config()
    _check(lib().bcs_config_default(ct.byref(c)))
    for k, v in overrides.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


def bcs_create(n, cfg=None, stream=None):
    h = _vp()
    st = lib().bcs_create(ct.byref(h), n, ct.byref(cfg) if cfg is not None else None,
                          stream if stream is not None else _current_stream())
    _check(st)
    _dims[_key(h)] = [int(n), 0, 0]
    return h


def bcs_destroy(h):
    _dims.pop(_key(h), None)
    return lib().bcs_destroy(h)


def bcs_set_config(h, cfg):
    return _check(lib().bcs_set_config(h, ct.byref(cfg)), h)


def bcs_set_structure(h, n_cells, owner, neighbour):
    _solver_dims(h)
    F = len(owner)
    (po, pn), mem = _marshal((owner, "int32", F), (neighbour, "int32", F))
    _check(lib().bcs_set_structure(h, n_cells, F, po, pn, mem), h)
    _dims[_key(h)][1:] = [int(n_cells), F]
    return BCS_OK


def bcs_set_values(h, diag, upper, lower):
    n, C, F = _solver_dims(h)
    (pd, pu, pl), mem = _marshal((diag, "float64", _cnt(C, n, n)), (upper, "float64", _cnt(F, n, n)),
                                 (lower, "float64", _cnt(F, n, n)))
    return _check(lib().bcs_set_values(h, pd, pu, pl, mem), h)


def bcs_flow_params_default(**overrides):
    p = bcs_flow_params()
    _check(lib().bcs_flow_params_default(ct.byref(p)))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def bcs_assemble_density(h, Q, area, normal, dist, prm, diag=None, upper=None, lower=None):
    n, C, F = _solver_dims(h)
    f = "float64"
    (pq, pa, pn, pd, pdg, pu, pl), mem = _marshal((Q, f, _cnt(C, 5)), (area, f, F), (normal, f, _cnt(F, 3)),
                                                  (dist, f, F), (diag, f, _cnt(C, 25)), (upper, f, _cnt(F, 25)),
                                                  (lower, f, _cnt(F, 25)))
    return _check(lib().bcs_assemble_density(h, pq, pa, pn, pd, ct.byref(prm), pdg, pu, pl, mem), h)


def _ints(vals):
    return (ct.c_int * len(vals))(*vals)


def bcs_pack_vector(h, ncomp, fields, out):
    n, C, F = _solver_dims(h)
    if len(fields) != len(ncomp):
        raise ValueError("one field per entry of ncomp")
    ptrs, mem = _marshal(*((a, "float64", _cnt(C, m)) for a, m in zip(fields, ncomp)), (out, "float64", _cnt(C, n)))
    arr = (ct.c_void_p * len(fields))(*ptrs[:-1])
    return _check(lib().bcs_pack_vector(h, len(ncomp), _ints(ncomp), arr, ptrs[-1], mem), h)


def bcs_unpack_vector(h, ncomp, vec, fields):
    n, C, F = _solver_dims(h)
    if len(fields) != len(ncomp):
        raise ValueError("one field per entry of ncomp")
    ptrs, mem = _marshal((vec, "float64", _cnt(C, n)), *((a, "float64", _cnt(C, m)) for a, m in zip(fields, ncomp)))
    arr = (ct.c_void_p * len(fields))(*ptrs[1:])
    return _check(lib().bcs_unpack_vector(h, len(ncomp), _ints(ncomp), ptrs[0], arr, mem), h)


def bcs_pack_coefficients(h, ncomp, coupling, diag=None, upper=None, lower=None):
    """coupling[a][b] = (diag, upper, lower) arrays or None (zero coupling)."""
    n, C, F = _solver_dims(h)
    nf = len(ncomp)
    if len(coupling) != nf or any(len(row) != nf for row in coupling):
        raise ValueError("coupling must be an nfields x nfields table")
    specs = []
    for a in range(nf):
        for b in range(nf):
            cp = coupling[a][b]
            if cp is not None:
                if len(cp) != 3:
                    raise ValueError("a coupling is (diag, upper, lower)")
                m = ncomp[a] * ncomp[b]
                specs += [(cp[0], "float64", _cnt(C, m)), (cp[1], "float64", _cnt(F, m)), (cp[2], "float64", _cnt(F, m))]
    flat = [sp[0] for sp in specs]
    ptrs, mem = _marshal(*specs, (diag, "float64", _cnt(C, n, n)), (upper, "float64", _cnt(F, n, n)),
                         (lower, "float64", _cnt(F, n, n)))
    tab = (bcs_coupling * (nf * nf))()
    it = iter(ptrs[:len(flat)])
    for a in range(nf):
        for b in range(nf):
            if coupling[a][b] is not None:
                tab[a * nf + b] = bcs_coupling(next(it), next(it), next(it))
    pd, pu, pl = ptrs[len(flat):]
    return _check(lib().bcs_pack_coefficients(h, nf, _ints(ncomp), tab, pd, pu, pl, mem), h)


def bcs_invalidate_hierarchy(h):
    return _check(lib().bcs_invalidate_hierarchy(h), h)


def bcs_solve(h, b, x, check=False):
    """Solve in place into x; returns (status, result dict)."""
    n, C, F = _solver_dims(h)
    (pb, px), mem = _marshal((b, "float64", _cnt(C, n)), (x, "float64", _cnt(C, n)))
    res = bcs_result()
    st = lib().bcs_solve(h, pb, px, mem, ct.byref(res))
    if st in (BCS_EINVAL, BCS_ENOMEM, BCS_ECUDA, BCS_ESTATE) or (check and st != BCS_OK):
        _check(st, h)
    return st, res.as_dict()


def bcs_solve_batch(handles, bs, xs):
    """Solve len(handles) systems together (in place into xs[i]); returns
    (status, [result dict per system])."""
    k = len(handles)
    if not (len(bs) == len(xs) == k):
        raise ValueError("one right-hand side and one solution per solver")
    specs = []
    for h, b, x in zip(handles, bs, xs):
        n, C, F = _solver_dims(h)
        specs += [(b, "float64", _cnt(C, n)), (x, "float64", _cnt(C, n))]
    ptrs, mem = _marshal(*specs)
    hs = (_vp * k)(*[h.value if isinstance(h, ct.c_void_p) else h for h in handles])
    pb = (_vp * k)(*ptrs[0::2])
    px = (_vp * k)(*ptrs[1::2])
    res = (bcs_result * k)()
    st = lib().bcs_solve_batch(hs, k, pb, px, mem, res)
    if st in (BCS_EINVAL, BCS_ENOMEM, BCS_ECUDA, BCS_ESTATE):
        _check(st, handles[0])
    return st, [r.as_dict() for r in res]


def solve_batch(solvers, bs, xs=None):
    """Solver objects' systems solved together: (xs, status, results)."""
    if xs is None:
        xs = [np.zeros_like(b) if isinstance(b, np.ndarray) else b.new_zeros(b.shape) for b in bs]
    st, res = bcs_solve_batch([s.h for s in solvers], bs, xs)
    return xs, st, res


def bcs_spmv(h, x, y):
    n, C, F = _solver_dims(h)
    (px, py), mem = _marshal((x, "float64", _cnt(C, n)), (y, "float64", _cnt(C, n)))
    return _check(lib().bcs_spmv(h, px, py, mem), h)


def bcs_precond_apply(h, v, z):
    n, C, F = _solver_dims(h)
    (pv, pz), mem = _marshal((v, "float64", _cnt(C, n)), (z, "float64", _cnt(C, n)))
    return _check(lib().bcs_precond_apply(h, pv, pz, mem), h)


def bcs_get_bsr(h, C, F, n, nnz, values=True):
    rp = np.zeros(C + 1, np.int32)
    col = np.zeros(nnz, np.int32)
    val = np.zeros((nnz, n, n)) if values else None
    pd = np.zeros(C, np.int32)
    pu = np.zeros(max(F, 1), np.int32)
    pl = np.zeros(max(F, 1), np.int32)
    _check(lib().bcs_get_bsr(h, rp.ctypes.data, col.ctypes.data, val.ctypes.data if values else None,
                             pd.ctypes.data, pu.ctypes.data, pl.ctypes.data), h)
    return dict(rows=C, n=n, row_ptr=rp, col=col, val=val, pos_diag=pd, pos_up=pu[:F], pos_lo=pl[:F])


def bcs_num_levels(h):
    return lib().bcs_num_levels(h)


def bcs_get_level_info(h, l):
    r, nz, pn, k = ct.c_int(), ct.c_int(), ct.c_int(), ct.c_int()
    _check(lib().bcs_get_level_info(h, l, ct.byref(r), ct.byref(nz), ct.byref(pn), ct.byref(k)), h)
    return dict(rows=r.value, nnz=nz.value, p_nnz=pn.value, coarse_kind=k.value)


def bcs_get_level(h, l, n):
    i = bcs_get_level_info(h, l)
    rp = np.zeros(i["rows"] + 1, np.int32)
    col = np.zeros(i["nnz"], np.int32)
    val = np.zeros((i["nnz"], n, n))
    agg = np.full(i["rows"], -1, np.int32)
    dinv = np.zeros((i["rows"], n, n))
    _check(lib().bcs_get_level(h, l, rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                               agg.ctypes.data if i["coarse_kind"] < 0 else None, dinv.ctypes.data), h)
    return dict(rows=i["rows"], n=n, row_ptr=rp, col=col, val=val, agg=agg, dinv=dinv,
                coarse_kind=i["coarse_kind"])


def bcs_get_prolongation(h, l, n):
    i = bcs_get_level_info(h, l)
    rp = np.zeros(i["rows"] + 1, np.int32)
    col = np.zeros(i["p_nnz"], np.int32)
    val = np.zeros((i["p_nnz"], n, n))
    om = ct.c_double()
    _check(lib().bcs_get_prolongation(h, l, rp.ctypes.data, col.ctypes.data, val.ctypes.data, ct.byref(om)), h)
    return dict(rows=i["rows"], n=n, row_ptr=rp, col=col, val=val, omega=om.value)


def bcs_get_dilu(h, l, rows, n):
    """(ncolours, colour[rows], einv[rows][n][n]) of level l, or (-1, None, None)."""
    nc = ct.c_int()
    col = np.zeros(rows, np.int32)
    einv = np.zeros((rows, n, n))
    _check(lib().bcs_get_dilu(h, l, ct.byref(nc), col.ctypes.data, einv.ctypes.data), h)
    return (nc.value, col, einv) if nc.value > 0 else (-1, None, None)


def bcs_get_coarse_inverse(h, N):
    out = np.zeros((N, N))
    _check(lib().bcs_get_coarse_inverse(h, out.ctypes.data), h)
    return out


def bcs_get_stats(h):
    st = bcs_stats()
    _check(lib().bcs_get_stats(h, ct.byref(st)), h)
    kinds = {}
    for k in range(NUM_KERNEL_KINDS):
        name = lib().bcs_kernel_kind_name(k).decode()
        if name:
            kinds[name] = dict(launches=st.kind_launches[k], ms=st.kind_ms[k], bytes=st.kind_bytes[k],
                               flops=st.kind_flops[k])
    return dict(launches=st.launches, kinds=kinds)


def bcs_get_kernel_times(h):
    """{kernel name: dict(launches, ms, bytes, kind)} (profile = 1)."""
    buf = ct.create_string_buffer(1 << 20)
    _check(lib().bcs_get_kernel_times(h, buf, len(buf)), h)
    out = {}
    for line in buf.value.decode().splitlines():
        name, n, ms, b, kind = line.split("\t")
        out[name] = dict(launches=int(n), ms=float(ms), bytes=float(b), kind=int(kind))
    return out


def bcs_get_level_times(h, level):
    """{kind name: dict(launches, ms, bytes)} of the timed launches on one
    hierarchy level (profile = 1); kinds without a launch are left out."""
    n = (ct.c_longlong * NUM_KERNEL_KINDS)()
    ms = (ct.c_double * NUM_KERNEL_KINDS)()
    b = (ct.c_double * NUM_KERNEL_KINDS)()
    _check(lib().bcs_get_level_times(h, int(level), ct.cast(n, _vp), ct.cast(ms, _vp), ct.cast(b, _vp)), h)
    return {bcs_kernel_kind_name(k): dict(launches=n[k], ms=ms[k], bytes=b[k])
            for k in range(NUM_KERNEL_KINDS) if n[k] > 0}


def bcs_reset_stats(h):
    return _check(lib().bcs_reset_stats(h), h)


def bcs_kernel_kind_name(k):
    return lib().bcs_kernel_kind_name(k).decode()


def kind_mask(*names):
    """profile_kinds bitmask for the kernel kinds with these names."""
    table = {bcs_kernel_kind_name(k): k for k in range(NUM_KERNEL_KINDS)}
    return sum(1 << table[nm] for nm in names)


def bcs_last_error(h):
    return lib().bcs_last_error(h).decode()


def bcs_device_bytes(h):
    return lib().bcs_device_bytes(h)


def bcs_ldu_structure_noalloc(n_cells, owner, neighbour, row_ptr, col, pos_diag, pos_up, pos_lo, stream=None):
    """Allocation-free structure build into caller-provided CUDA tensors.

    Returns (status, message); the library allocates no device memory here.
    """
    C, F, i = int(n_cells), len(owner), "int32"
    sized = 1 <= C <= (1 << 20)   # beyond the limit the library answers BCS_EINVAL by itself
    (po, pn, prp, pc, pd, pu, pl), mem = _marshal(
        (owner, i, F), (neighbour, i, F), (row_ptr, i, C + 1 if sized else None),
        (col, i, C + 2 * F if sized else None), (pos_diag, i, C if sized else None), (pos_up, i, F),
        (pos_lo, i, F))
    if mem != BCS_MEM_DEVICE:
        raise ValueError("bcs_ldu_structure_noalloc takes device arrays only")
    buf = ct.create_string_buffer(256)
    st = lib().bcs_ldu_structure_noalloc(n_cells, F, po, pn, prp, pc, pd, pu, pl,
                                         stream if stream is not None else _current_stream(), buf, 256)
    return st, buf.value.decode()


def torch_allocator():
    """(alloc, release) callbacks drawing the solver's device memory from
    PyTorch's caching allocator on the solver's stream."""
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(nbytes, stream=stream or 0)
        except RuntimeError:
            return None

    def _release(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    return ALLOC_FN(_alloc), RELEASE_FN(_release)


class Solver:
    """Owning wrapper: a solver handle for n x n blocks. allocator="torch"
    takes the device memory from PyTorch's caching allocator."""

    def __init__(self, n, allocator=None, **cfg):
        self.n = n
        self.cfg = bcs_config_default(**cfg)
        self._alloc_cbs = None
        if allocator == "torch":
            self._alloc_cbs = torch_allocator()
            self.cfg.alloc, self.cfg.release = self._alloc_cbs
        elif allocator is not None:
            raise ValueError("allocator: None or 'torch'")
        self.h = bcs_create(n, self.cfg)
        self.C = self.F = 0

    def close(self):
        if getattr(self, "h", None):
            bcs_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_config(self, **cfg):
        for k, v in cfg.items():
            setattr(self.cfg, k, v)
        bcs_set_config(self.h, self.cfg)

    def set_structure(self, n_cells, owner, neighbour):
        """LDU face addressing (int32 owner / neighbour per face, Sec. 2.3):
        builds the block-CSR structure; drops any values and hierarchy."""
        self.C, self.F = int(n_cells), len(owner)
        bcs_set_structure(self.h, n_cells, owner, neighbour)

    def set_values(self, diag, upper, lower):
        """Coefficients diag[C][n][n], upper / lower[F][n][n] (FP64): full AMG
        setup the first time, values-only resetup afterwards (Alg. 1)."""
        bcs_set_values(self.h, diag, upper, lower)

    def load(self, system, device=None):
        """Structure + values of a synth system dict (numpy; device=torch device copies first)."""
        keys = ("owner", "neighbour", "diag", "upper", "lower")
        arr = {k: system[k] for k in keys}
        if device is not None:
            import torch
            arr = {k: torch.from_numpy(np.ascontiguousarray(v)).to(device) for k, v in arr.items()}
        self.set_structure(system["n_cells"], arr["owner"], arr["neighbour"])
        self.set_values(arr["diag"], arr["upper"], arr["lower"])

    def _like(self, ref, shape):
        return np.zeros(shape) if isinstance(ref, np.ndarray) else ref.new_zeros(shape)

    def pack_vector(self, fields, ncomp):
        """Block AoS vector [C][n] from segregated fields (Alg. 1 step 1)."""
        out = self._like(fields[0], (self.C, self.n))
        bcs_pack_vector(self.h, ncomp, fields, out)
        return out

    def unpack_vector(self, vec, ncomp):
        """Segregated fields from a block AoS vector (Alg. 1 step 15)."""
        fields = [self._like(vec, (self.C * m,)) for m in ncomp]
        bcs_unpack_vector(self.h, ncomp, vec, fields)
        return fields

    def pack_coefficients(self, coupling, ncomp, to_values=False):
        """LDU blocks (diag, upper, lower) from field couplings (Alg. 1 step
        5), or straight into the solver's values followed by setup."""
        if to_values:
            bcs_pack_coefficients(self.h, ncomp, coupling)
            return None
        ref = next(a for row in coupling for cp in row if cp is not None for a in cp)
        n = self.n
        out = (self._like(ref, (self.C, n, n)), self._like(ref, (self.F, n, n)), self._like(ref, (self.F, n, n)))
        bcs_pack_coefficients(self.h, ncomp, coupling, *out)
        return out

    def permutation(self):
        """The caller's cell of every internal row (identity without reorder)."""
        perm = np.zeros(self.C, np.int32)
        _check(lib().bcs_get_permutation(self.h, perm.ctypes.data), self.h)
        return perm

    def assemble_density(self, Q, area, normal, dist, to_values=False, **prm):
        """Density-based system from cell states and face geometry (Sec. 2.1).
        to_values: write the solver's own values and set up (as set_values);
        otherwise return (diag, upper, lower) in the inputs' memory space."""
        p = bcs_flow_params_default(**prm)
        if to_values:
            bcs_assemble_density(self.h, Q, area, normal, dist, p)
            return None
        C, F = self.C, self.F
        if isinstance(Q, np.ndarray):
            out = [np.zeros((C, 5, 5)), np.zeros((F, 5, 5)), np.zeros((F, 5, 5))]
        else:
            out = [Q.new_zeros((C, 5, 5)), Q.new_zeros((F, 5, 5)), Q.new_zeros((F, 5, 5))]
        bcs_assemble_density(self.h, Q, area, normal, dist, p, *out)
        return tuple(out)

    def solve(self, b, x=None):
        """Solve A x = b to cfg.tol (x holds x0 on entry, zeros when None);
        returns (x, status, result dict)."""
        if x is None:
            x = np.zeros_like(b) if isinstance(b, np.ndarray) else b.new_zeros(b.shape)
        st, res = bcs_solve(self.h, b, x)
        return x, st, res

    def spmv(self, x, y=None):
        """y = A x with the fine FP64 matrix."""
        if y is None:
            y = np.zeros_like(x) if isinstance(x, np.ndarray) else x.new_zeros(x.shape)
        bcs_spmv(self.h, x, y)
        return y

    def precond(self, v, z=None):
        """z = M^-1 v: one application of the configured preconditioner."""
        if z is None:
            z = np.zeros_like(v) if isinstance(v, np.ndarray) else v.new_zeros(v.shape)
        bcs_precond_apply(self.h, v, z)
        return z

    def bsr(self, values=True):
        return bcs_get_bsr(self.h, self.C, self.F, self.n, self.C + 2 * self.F, values)

    @property
    def levels(self):
        return bcs_num_levels(self.h)

    def level(self, l):
        return bcs_get_level(self.h, l, self.n)

    def level_info(self, l):
        return bcs_get_level_info(self.h, l)

    def prolongation(self, l):
        return bcs_get_prolongation(self.h, l, self.n)

    def dilu(self, l):
        return bcs_get_dilu(self.h, l, self.level_info(l)["rows"], self.n)

    def coarse_inverse(self):
        info = self.level_info(self.levels - 1)
        return bcs_get_coarse_inverse(self.h, info["rows"] * self.n)

    def stats(self):
        return bcs_get_stats(self.h)

    def reset_stats(self):
        bcs_reset_stats(self.h)

    def kernel_times(self):
        return bcs_get_kernel_times(self.h)

    def level_times(self):
        """[per level {kind name: dict(launches, ms, bytes)}] (profile = 1)."""
        return [bcs_get_level_times(self.h, l) for l in range(self.levels)]


# ---------------------------------------------------------------- serving
def bcs_server_create(budget_bytes=0, slots=4, cfg=None):
    h = _vp()
    _check(lib().bcs_server_create(ct.byref(h), budget_bytes, slots, ct.byref(cfg) if cfg is not None else None))
    return h


def bcs_server_destroy(h):
    k = _key(h)
    for key in [key for key in _dims if isinstance(key, tuple) and key[0] == k]:
        del _dims[key]
    return lib().bcs_server_destroy(h)


def bcs_server_register_case(h, n, n_cells, owner, neighbour):
    owner = np.ascontiguousarray(owner, np.int32)
    neighbour = np.ascontiguousarray(neighbour, np.int32)
    if owner.size != neighbour.size:
        raise ValueError("owner and neighbour must have one entry per face")
    cid = ct.c_int()
    _check(lib().bcs_server_register_case(h, n, n_cells, owner.size, owner.ctypes.data, neighbour.ctypes.data,
                                          ct.byref(cid)))
    _dims[(_key(h), cid.value)] = [int(n), int(n_cells), int(owner.size)]
    return cid.value


def bcs_server_submit(h, case_id, diag, upper, lower, b, x):
    """numpy arrays (host) or CUDA tensors (device), all five alike; they must
    stay alive until the request completes."""
    t = ct.c_int64()
    d = _dims.get((_key(h), case_id))
    if d is None:
        raise ValueError(f"case {case_id} is not registered with this server")
    n, C, F = d
    f = "float64"
    ptrs, mem = _marshal((diag, f, C * n * n), (upper, f, F * n * n), (lower, f, F * n * n), (b, f, C * n),
                         (x, f, C * n))
    _check(lib().bcs_server_submit(h, case_id, *ptrs, mem, ct.byref(t)))
    return t.value


def bcs_server_wait(h, ticket, timeout_ms=-1):
    res = bcs_result()
    lat = ct.c_double()
    st = lib().bcs_server_wait(h, ticket, timeout_ms, ct.byref(res), ct.byref(lat))
    return st, res.as_dict(), lat.value


def bcs_server_get_stats(h):
    st = bcs_server_stats()
    _check(lib().bcs_server_get_stats(h, ct.byref(st)))
    return st.as_dict()


def bcs_server_reset_stats(h):
    return _check(lib().bcs_server_reset_stats(h))


class Server:
    """Owning wrapper of a serving instance; keeps submitted arrays alive."""

    def __init__(self, budget_bytes=0, slots=4, batch=1, **cfg):
        self.h = bcs_server_create(budget_bytes, slots, bcs_config_default(**cfg))
        self._keep = {}
        if batch != 1:
            _check(lib().bcs_server_set_batch(self.h, batch))

    def close(self):
        if getattr(self, "h", None):
            bcs_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def register(self, system):
        return bcs_server_register_case(self.h, system["n"], system["n_cells"], system["owner"],
                                        system["neighbour"])

    def submit(self, case_id, system, x=None):
        """system: dict of numpy arrays or of CUDA tensors (diag, upper,
        lower, b); x: initial guess of the same kind (zeros when None)."""
        arrs = [system[k] for k in ("diag", "upper", "lower", "b")]
        if isinstance(arrs[0], np.ndarray):
            arrs = [np.ascontiguousarray(a, np.float64) for a in arrs]
            if x is None:
                x = np.zeros_like(arrs[3])
        else:
            if x is None:
                x = arrs[3].new_zeros(arrs[3].shape)
            # the request runs on the case's own stream, which does not wait
            # for the caller's: the arrays (and the zeros just queued) must be
            # complete when the request is submitted
            import torch
            torch.cuda.current_stream(arrs[3].device).synchronize()
        t = bcs_server_submit(self.h, case_id, *arrs, x)
        self._keep[t] = (arrs, x)
        return t

    def wait(self, ticket, timeout_ms=-1):
        st, res, lat = bcs_server_wait(self.h, ticket, timeout_ms)
        if st == BCS_TIMEOUT:
            return st, res, lat, None
        arrs, x = self._keep.pop(ticket)
        return st, res, lat, x

    def reset_stats(self):
        _check(lib().bcs_server_reset_stats(self.h))

    def stats(self):
        return bcs_server_get_stats(self.h)

    def last_error(self):
        """Message of the most recent failed request ("" when none failed)."""
        buf = ct.create_string_buffer(1024)
        lib().bcs_server_last_error(self.h, buf, len(buf))
        return buf.value.decode()
