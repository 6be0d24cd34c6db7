"""Python binding of the C ABI in include/amg.h (argument marshalling only).

Every function has the name of the C entry point it calls.  Arrays may be numpy arrays
(host memory) or torch tensors (host or CUDA); pointers are passed through unchanged and
all arithmetic runs in libamg_gb300.so.  There is no fallback: if the library is missing
or fails to load, the import of this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

AMG_OK, AMG_ERR_INVALID_ARG, AMG_ERR_OOM, AMG_ERR_CUDA, AMG_ERR_ZERO_DIAG, AMG_ERR_EIGEN, \
    AMG_ERR_COARSE_NOT_SPD, AMG_ERR_NOT_CONVERGED, AMG_ERR_BUDGET, AMG_ERR_UNSUPPORTED, AMG_ERR_INTERNAL, \
    AMG_PENDING = range(12)
AMG_VAR_1NORM, AMG_VAR_OFFLMP, AMG_VAR_SPRSFY, AMG_VAR_CNSTRNT = 1, 2, 4, 8
AMG_FP64, AMG_MIXED = 0, 1
AMG_PT_ORTHONORMAL, AMG_PT_UNIT = 0, 1
AMG_LAMBDA_ONE, AMG_LAMBDA_POWER = 0, 1
AMG_STRENGTH_MATRIX, AMG_STRENGTH_DISTANCE = 0, 1
AMG_KRYLOV_CG, AMG_KRYLOV_GMRES = 0, 1
AMG_LAYOUT_AUTO, AMG_LAYOUT_CSR, AMG_LAYOUT_SELL = 0, 1, 2
AMG_COARSE_AUTO, AMG_COARSE_INVERSE = 0, 1
PHASES = ("input", "strength", "aggregate", "filter", "eigen", "prolong", "galerkin_ap", "galerkin_rap",
          "smoother", "coarse", "prepare")
EXPORTS = {"A.rp": (0, np.int64), "A.ci": (1, np.int32), "A.v": (2, np.float64), "strong": (3, np.uint8),
           "removed": (4, np.uint8), "lumpflag": (5, np.uint8), "Abar.rp": (6, np.int64), "Abar.ci": (7, np.int32),
           "Abar.v": (8, np.float64), "agg": (9, np.int32), "root": (10, np.uint8), "P.rp": (11, np.int64),
           "P.ci": (12, np.int32), "P.v": (13, np.float64), "R.rp": (14, np.int64), "R.ci": (15, np.int32),
           "R.v": (16, np.float64), "Dsm": (17, np.float64), "scalars": (18, np.float64), "B": (19, np.float64),
           "cflag": (20, np.uint8), "coords": (21, np.float64)}


class AmgError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: status {status} ({detail})")


class amg_csr_t(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("on_device", C.c_int)]


class amg_params_t(C.Structure):
    _fields_ = [("theta", C.c_double), ("variants", C.c_uint), ("tau", C.c_double), ("sigma", C.c_double),
                ("cheb_degree", C.c_int), ("cheb_ratio", C.c_double), ("cheb_boost", C.c_double),
                ("power_iters", C.c_int),
                ("max_coarse", C.c_int), ("max_levels", C.c_int), ("precision", C.c_int), ("pt_scaling", C.c_int),
                ("onenorm_lambda", C.c_int), ("max_iter", C.c_int), ("seed", C.c_uint64),
                ("lambda_override", C.c_double), ("cuda_stream", C.c_void_p), ("strength", C.c_int),
                ("trace", C.c_int), ("krylov", C.c_int), ("restart", C.c_int), ("spmv_layout", C.c_int),
                ("block_size", C.c_int), ("nullspace_dim", C.c_int), ("coarse_solve", C.c_int)]


class amg_info_t(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("relres_true", C.c_double), ("setup_ms", C.c_double),
                ("solve_ms", C.c_double), ("levels", C.c_int), ("op_complexity", C.c_double)]


class amg_dcsr_t(C.Structure):
    _fields_ = [("nrow", C.c_int64), ("ncol", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class amg_server_config_t(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("setup_threads", C.c_int), ("max_systems", C.c_int),
                ("max_rows", C.c_int64), ("tol", C.c_double), ("tune", C.c_int), ("params", amg_params_t)]


class amg_request_info_t(C.Structure):
    _fields_ = [("status", C.c_int), ("nrhs", C.c_int), ("iters_max", C.c_int), ("cache_hit", C.c_int),
                ("relres_max", C.c_double), ("queue_ms", C.c_double), ("setup_ms", C.c_double),
                ("latency_ms", C.c_double)]


class amg_server_stats_t(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("solves", C.c_int64),
                ("cache_hits", C.c_int64), ("cache_misses", C.c_int64), ("evictions", C.c_int64),
                ("failed", C.c_int64), ("iterations", C.c_int64), ("commits", C.c_int64),
                ("engine_busy_ms", C.c_double), ("bytes_hierarchies", C.c_size_t), ("bytes_engine", C.c_size_t),
                ("resident_hierarchies", C.c_int), ("first_error", C.c_char * 256)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_2103_10476_gb300.build.build() first")
    L = C.CDLL(LIB_PATH)
    vp, st = C.c_void_p, C.c_int
    sig = {
        "amg_params_default": (None, [C.POINTER(amg_params_t)]),
        "amg_setup": (st, [C.POINTER(amg_csr_t), vp, C.POINTER(amg_params_t), C.POINTER(vp)]),
        "amg_setup_coords": (st, [C.POINTER(amg_csr_t), vp, vp, C.c_int, C.POINTER(amg_params_t), C.POINTER(vp)]),
        "amg_solve": (st, [vp, vp, vp, C.c_double, C.POINTER(amg_info_t)]),
        "amg_solve_multi": (st, [vp, C.c_int, vp, vp, C.c_double, C.POINTER(amg_info_t)]),
        "amg_free": (st, [vp]),
        "amg_num_levels": (st, [vp, C.POINTER(C.c_int)]),
        "amg_coarse_solver": (st, [vp, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.POINTER(C.c_double)]),
        "amg_setup_trace": (st, [vp, C.c_int, C.POINTER(C.c_double)]),
        "amg_level_info": (st, [vp, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "amg_export_count": (st, [vp, C.c_int, C.c_int, C.POINTER(C.c_int64)]),
        "amg_export": (st, [vp, C.c_int, C.c_int, vp]),
        "amg_vcycle": (st, [vp, vp, vp]),
        "amg_spgemm": (st, [C.POINTER(amg_csr_t), C.c_int64, C.POINTER(amg_csr_t), C.c_int64, vp,
                            C.POINTER(amg_dcsr_t)]),
        "amg_csr_release": (st, [C.POINTER(amg_dcsr_t)]),
        "amg_spgemm_noalloc": (st, [C.POINTER(amg_csr_t), C.c_int64, C.POINTER(amg_csr_t), C.c_int64, vp, vp, vp, vp,
                                    C.c_int64, C.POINTER(C.c_int64)]),
        "amg_dcsr_download": (st, [C.POINTER(amg_dcsr_t), vp, vp, vp]),
        "amg_launch_count": (C.c_int64, []),
        "amg_profile_enable": (st, [C.c_int]),
        "amg_profile_read": (st, [C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "amg_setup_batch": (st, [C.c_int, C.POINTER(C.POINTER(amg_csr_t)), C.POINTER(vp), C.POINTER(amg_params_t),
                                 C.c_int, C.POINTER(vp)]),
        "amg_batch_create": (st, [C.c_int, C.POINTER(vp), vp, C.c_int, C.POINTER(vp)]),
        "amg_batch_solve": (st, [vp, C.POINTER(vp), C.POINTER(vp), C.c_double, C.POINTER(amg_info_t)]),
        "amg_batch_free": (st, [vp]),
        "amg_solve_batch": (st, [C.c_int, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.c_double,
                                 C.POINTER(amg_info_t)]),
        "amg_batch_info": (st, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int64),
                                C.POINTER(C.c_int64)]),
        "amg_server_config_default": (None, [C.POINTER(amg_server_config_t)]),
        "amg_server_create": (st, [C.POINTER(amg_server_config_t), C.POINTER(vp)]),
        "amg_server_submit": (st, [vp, C.POINTER(amg_csr_t), C.c_int, vp, vp, C.POINTER(C.c_uint64)]),
        "amg_server_poll": (st, [vp, C.c_uint64, C.POINTER(amg_request_info_t)]),
        "amg_server_wait": (st, [vp, C.c_uint64, C.POINTER(amg_request_info_t)]),
        "amg_server_stats": (st, [vp, C.POINTER(amg_server_stats_t)]),
        "amg_server_destroy": (st, [vp]),
        "amg_router_create": (st, [C.c_int, C.POINTER(vp)]),
        "amg_router_route": (st, [vp, C.POINTER(amg_csr_t), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_uint64),
                                  C.POINTER(C.c_int)]),
        "amg_router_attach": (st, [vp, C.c_int, vp]),
        "amg_router_submit": (st, [vp, C.POINTER(amg_csr_t), C.c_int, vp, vp, C.POINTER(C.c_uint64),
                                   C.POINTER(C.c_int)]),
        "amg_router_poll": (st, [vp, C.c_uint64, C.POINTER(amg_request_info_t), C.POINTER(C.c_int)]),
        "amg_router_wait": (st, [vp, C.c_uint64, C.POINTER(amg_request_info_t), C.POINTER(C.c_int)]),
        "amg_router_stats": (st, [vp, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_double)]),
        "amg_router_destroy": (st, [vp]),
        "amg_status_string": (C.c_char_p, [st]),
        "amg_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


def _ptr(a):
    """(pointer, on_device) of a numpy array or torch tensor (must be contiguous)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), int(a.is_cuda)
    raise TypeError(f"unsupported array type {type(a)}")


def _check(status: int, where: str):
    if status != AMG_OK:
        raise AmgError(status, where, lib.amg_last_error().decode(errors="replace"))


def csr_arg(n: int, row_ptr, col, val) -> amg_csr_t:
    rp, d0 = _ptr(row_ptr)
    ci, d1 = _ptr(col)
    v, d2 = _ptr(val)
    if len({d0, d1, d2}) != 1:
        raise ValueError("row_ptr, col and val must live on the same side")
    nnz = int(row_ptr[-1])
    return amg_csr_t(n, nnz, rp, ci, v, d0)


def amg_params_default(**overrides) -> amg_params_t:
    p = amg_params_t()
    lib.amg_params_default(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def amg_setup(A: amg_csr_t, nullspace=None, params: amg_params_t | None = None):
    """Returns the handle (a c_void_p); raises AmgError with the library status on failure."""
    p = params if params is not None else amg_params_default()
    h = C.c_void_p()
    ns, _ = _ptr(nullspace)
    _check(lib.amg_setup(C.byref(A), ns, C.byref(p), C.byref(h)), "amg_setup")
    return h


def amg_setup_coords(A: amg_csr_t, nullspace=None, coords=None, params: amg_params_t | None = None):
    """amg_setup with row coordinates (n x dim array, host or device, same side as A), for the
    distance-Laplacian strength; raises AmgError on failure."""
    p = params if params is not None else amg_params_default()
    h = C.c_void_p()
    ns, _ = _ptr(nullspace)
    xc, _ = _ptr(coords)
    dim = 0 if coords is None else (1 if len(coords.shape) == 1 else int(coords.shape[1]))
    _check(lib.amg_setup_coords(C.byref(A), ns, xc, dim, C.byref(p), C.byref(h)), "amg_setup_coords")
    return h


def amg_setup_status(A: amg_csr_t, nullspace=None, params: amg_params_t | None = None):
    """(handle or None, status) without raising."""
    p = params if params is not None else amg_params_default()
    h = C.c_void_p()
    ns, _ = _ptr(nullspace)
    s = lib.amg_setup(C.byref(A), ns, C.byref(p), C.byref(h))
    return (h if s == AMG_OK else None), s


def amg_solve(h, b, x, tol: float) -> amg_info_t:
    """Solves into x; returns the info struct (info.status holds NOT_CONVERGED if so)."""
    info = amg_info_t()
    pb, _ = _ptr(b)
    px, _ = _ptr(x)
    s = lib.amg_solve(h, pb, px, tol, C.byref(info))
    if s not in (AMG_OK, AMG_ERR_NOT_CONVERGED):
        _check(s, "amg_solve")
    info.status = s
    return info


def amg_solve_multi(h, B, X, tol: float):
    """k right-hand sides at once: B, X of shape (k, n) (numpy or torch, row j = column j of
    the C call).  Returns (status, [amg_info_t] * k)."""
    k = int(B.shape[0])
    infos = (amg_info_t * max(1, k))()
    pb, _ = _ptr(B)
    px, _ = _ptr(X)
    s = lib.amg_solve_multi(h, k, pb, px, tol, infos)
    if s not in (AMG_OK, AMG_ERR_NOT_CONVERGED):
        _check(s, "amg_solve_multi")
    return s, [infos[j] for j in range(k)]


def amg_free(h):
    _check(lib.amg_free(h), "amg_free")


def amg_num_levels(h) -> int:
    n = C.c_int()
    _check(lib.amg_num_levels(h, C.byref(n)), "amg_num_levels")
    return n.value


def amg_coarse_solver(h):
    """(degree, theta, delta, check) of the coarsest-level solve; degree 0: the dense inverse."""
    d, t, w, c = C.c_int(), C.c_double(), C.c_double(), C.c_double()
    _check(lib.amg_coarse_solver(h, C.byref(d), C.byref(t), C.byref(w), C.byref(c)), "amg_coarse_solver")
    return d.value, t.value, w.value, c.value


def amg_level_info(h, level: int):
    n, nnz, nagg = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib.amg_level_info(h, level, C.byref(n), C.byref(nnz), C.byref(nagg)), "amg_level_info")
    return n.value, nnz.value, nagg.value


def amg_export(h, level: int, what: str) -> np.ndarray:
    code, dt = EXPORTS[what]
    cnt = C.c_int64()
    _check(lib.amg_export_count(h, level, code, C.byref(cnt)), "amg_export_count")
    out = np.zeros(max(cnt.value, 1), dtype=dt)
    if cnt.value:
        _check(lib.amg_export(h, level, code, out.ctypes.data), "amg_export")
    return out[:cnt.value]


def amg_setup_trace(h, level: int) -> dict:
    """Setup phase times (ms) of one level of a hierarchy built with params.trace = 1."""
    ms = (C.c_double * len(PHASES))()
    _check(lib.amg_setup_trace(h, level, ms), "amg_setup_trace")
    return {name: ms[k] for k, name in enumerate(PHASES)}


def amg_vcycle(h, r, z):
    pr, _ = _ptr(r)
    pz, _ = _ptr(z)
    _check(lib.amg_vcycle(h, pr, pz), "amg_vcycle")


def amg_spgemm(A: amg_csr_t, ncolA: int, B: amg_csr_t, ncolB: int, stream=None):
    """C = A B on the device; returns host numpy (row_ptr, col, val)."""
    Cm = amg_dcsr_t()
    _check(lib.amg_spgemm(C.byref(A), ncolA, C.byref(B), ncolB, stream, C.byref(Cm)), "amg_spgemm")
    nrow, nnz = Cm.nrow, Cm.nnz
    try:
        rp = np.zeros(nrow + 1, dtype=np.int64)
        ci = np.zeros(max(nnz, 1), dtype=np.int32)
        v = np.zeros(max(nnz, 1), dtype=np.float64)
        _check(lib.amg_dcsr_download(C.byref(Cm), rp.ctypes.data, ci.ctypes.data, v.ctypes.data), "amg_dcsr_download")
    finally:
        lib.amg_csr_release(C.byref(Cm))
    return rp, ci[:nnz], v[:nnz]


KC_PCG_SPMV, KC_VCYCLE_SPMV, KC_SPGEMM = 0, 1, 2


def amg_launch_count() -> int:
    return int(lib.amg_launch_count())


def amg_profile_enable(on):
    """True/1: reset and record; 2: resume recording keeping the totals; False/0: stop."""
    _check(lib.amg_profile_enable(int(on)), "amg_profile_enable")


def amg_profile_read(kclass: int):
    """(launches, total_ms, total_bytes) of one timed kernel class."""
    n, ms, by = C.c_int64(), C.c_double(), C.c_double()
    _check(lib.amg_profile_read(kclass, C.byref(n), C.byref(ms), C.byref(by)), "amg_profile_read")
    return n.value, ms.value, by.value


def amg_spgemm_noalloc(A: amg_csr_t, ncolA: int, B: amg_csr_t, ncolB: int, C_row_ptr, C_col, C_val,
                       capacity: int, stream=None):
    """Allocation-free C = A B into caller-provided device arrays; returns (status, nnz(C))."""
    nnz = C.c_int64()
    prp, _ = _ptr(C_row_ptr)
    pci, _ = _ptr(C_col)
    pv, _ = _ptr(C_val)
    s = lib.amg_spgemm_noalloc(C.byref(A), ncolA, C.byref(B), ncolB, stream, prp, pci, pv, capacity, C.byref(nnz))
    return s, nnz.value


def _ptr_array(arrays):
    out = (C.c_void_p * max(1, len(arrays)))()
    for k, a in enumerate(arrays):
        out[k] = _ptr(a)[0]
    return out


def amg_setup_batch(As, nullspaces=None, params: amg_params_t | None = None, threads: int = 0):
    """List of handles, one per amg_csr_t in As (built concurrently); raises AmgError."""
    p = params if params is not None else amg_params_default()
    n = len(As)
    arr = (C.POINTER(amg_csr_t) * max(1, n))()
    for k, A in enumerate(As):
        arr[k] = C.pointer(A)
    ns = _ptr_array(nullspaces) if nullspaces is not None else None
    out = (C.c_void_p * max(1, n))()
    _check(lib.amg_setup_batch(n, arr, ns, C.byref(p), threads, out), "amg_setup_batch")
    return [C.c_void_p(out[k]) for k in range(n)]


def _handle_array(handles):
    arr = (C.c_void_p * max(1, len(handles)))()
    for k, h in enumerate(handles):
        arr[k] = h.value if isinstance(h, C.c_void_p) else h
    return arr


def amg_batch_create(handles, stream=None, tune: bool = False):
    bt = C.c_void_p()
    _check(lib.amg_batch_create(len(handles), _handle_array(handles), stream, int(tune), C.byref(bt)),
           "amg_batch_create")
    return bt


def amg_batch_solve(bt, bs, xs, tol: float):
    """Solves every system into xs[k]; returns (status, list of amg_info_t)."""
    n = len(bs)
    infos = (amg_info_t * max(1, n))()
    s = lib.amg_batch_solve(bt, _ptr_array(bs), _ptr_array(xs), tol, infos)
    if s not in (AMG_OK, AMG_ERR_NOT_CONVERGED):
        _check(s, "amg_batch_solve")
    return s, [infos[k] for k in range(n)]


def amg_batch_free(bt):
    _check(lib.amg_batch_free(bt), "amg_batch_free")


def amg_solve_batch(handles, bs, xs, tol: float):
    n = len(handles)
    infos = (amg_info_t * max(1, n))()
    s = lib.amg_solve_batch(n, _handle_array(handles), _ptr_array(bs), _ptr_array(xs), tol, infos)
    if s not in (AMG_OK, AMG_ERR_NOT_CONVERGED):
        _check(s, "amg_solve_batch")
    return s, [infos[k] for k in range(n)]


def amg_batch_info(bt):
    """(systems, levels, fine rows, kernels per replayed iteration)."""
    c, L, rows, gk = C.c_int(), C.c_int(), C.c_int64(), C.c_int64()
    _check(lib.amg_batch_info(bt, C.byref(c), C.byref(L), C.byref(rows), C.byref(gk)), "amg_batch_info")
    return c.value, L.value, rows.value, gk.value


def amg_server_config_default(params: amg_params_t | None = None, **overrides) -> amg_server_config_t:
    c = amg_server_config_t()
    lib.amg_server_config_default(C.byref(c))
    if params is not None:
        c.params = params
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


def amg_server_create(cfg: amg_server_config_t):
    srv = C.c_void_p()
    _check(lib.amg_server_create(C.byref(cfg), C.byref(srv)), "amg_server_create")
    return srv


def amg_server_submit(srv, A: amg_csr_t, nrhs: int, b, x) -> int:
    """Queues a request; b and x (nrhs * n doubles) and A's arrays must outlive it."""
    t = C.c_uint64()
    pb, _ = _ptr(b)
    px, _ = _ptr(x)
    _check(lib.amg_server_submit(srv, C.byref(A), nrhs, pb, px, C.byref(t)), "amg_server_submit")
    return t.value


def amg_server_poll(srv, ticket: int):
    """None while pending, else the request's amg_request_info_t."""
    info = amg_request_info_t()
    s = lib.amg_server_poll(srv, ticket, C.byref(info))
    if s == AMG_PENDING:
        return None
    _check(s, "amg_server_poll")
    return info


def amg_server_wait(srv, ticket: int) -> amg_request_info_t:
    info = amg_request_info_t()
    _check(lib.amg_server_wait(srv, ticket, C.byref(info)), "amg_server_wait")
    return info


def amg_server_stats(srv) -> amg_server_stats_t:
    st = amg_server_stats_t()
    _check(lib.amg_server_stats(srv, C.byref(st)), "amg_server_stats")
    return st


def amg_server_destroy(srv):
    _check(lib.amg_server_destroy(srv), "amg_server_destroy")


def amg_router_create(ndev: int):
    r = C.c_void_p()
    _check(lib.amg_router_create(ndev, C.byref(r)), "amg_router_create")
    return r


def amg_router_route(r, A: amg_csr_t, nrhs: int):
    """(device, content key, repeat) of a request for A with nrhs right-hand sides."""
    d, k, rep = C.c_int(), C.c_uint64(), C.c_int()
    _check(lib.amg_router_route(r, C.byref(A), nrhs, C.byref(d), C.byref(k), C.byref(rep)), "amg_router_route")
    return d.value, k.value, bool(rep.value)


def amg_router_attach(r, device: int, srv):
    _check(lib.amg_router_attach(r, device, srv), "amg_router_attach")


def amg_router_submit(r, A: amg_csr_t, nrhs: int, b, x):
    """(router ticket, device); b, x and A's arrays must outlive the request."""
    t, d = C.c_uint64(), C.c_int()
    pb, _ = _ptr(b)
    px, _ = _ptr(x)
    _check(lib.amg_router_submit(r, C.byref(A), nrhs, pb, px, C.byref(t), C.byref(d)), "amg_router_submit")
    return t.value, d.value


def amg_router_wait(r, ticket: int):
    """(amg_request_info_t, device that served it)."""
    info, d = amg_request_info_t(), C.c_int()
    _check(lib.amg_router_wait(r, ticket, C.byref(info), C.byref(d)), "amg_router_wait")
    return info, d.value


def amg_router_poll(r, ticket: int):
    """None while pending, else (amg_request_info_t, device)."""
    info, d = amg_request_info_t(), C.c_int()
    s = lib.amg_router_poll(r, ticket, C.byref(info), C.byref(d))
    if s == AMG_PENDING:
        return None
    _check(s, "amg_router_poll")
    return info, d.value


def amg_router_stats(r, device: int) -> dict:
    req, ops, rep, work = C.c_int64(), C.c_int64(), C.c_int64(), C.c_double()
    _check(lib.amg_router_stats(r, device, C.byref(req), C.byref(ops), C.byref(rep), C.byref(work)),
           "amg_router_stats")
    return {"requests": req.value, "operators": ops.value, "repeats": rep.value, "work": work.value}


def amg_router_destroy(r):
    _check(lib.amg_router_destroy(r), "amg_router_destroy")


def amg_status_string(s: int) -> str:
    return lib.amg_status_string(s).decode()


def amg_last_error() -> str:
    return lib.amg_last_error().decode(errors="replace")
