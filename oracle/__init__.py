"""CPU oracle of SA-AMG with the 1Norm / OffLmp / Cnstrnt / Sprsfy adaptations.

TEST INFRASTRUCTURE ONLY: the reference that the CUDA path is checked against.  Only the
tests, the smoke check and the benchmark's CPU-baseline / reference arm may import this
package.  It wraps `libsa_oracle.so` (plain single-threaded FP64 C, `sa_oracle.c`) through
ctypes and converts to and from numpy arrays.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sa_oracle.c")
LIB = os.path.join(HERE, "libsa_oracle.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_ZERO_DIAG, ERR_EIGEN, ERR_COARSE_NOT_SPD, ERR_NOT_CONVERGED, ERR_UNSUPPORTED = \
    0, 1, 2, 4, 5, 6, 7, 9
ONENORM, OFFLMP, SPRSFY, CNSTRNT = 1, 2, 4, 8


def build(force: bool = False) -> str:
    """Compile the oracle (no FMA contraction, so every product and sum rounds as written)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "sa_oracle.h"))):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", SRC,
                               "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class Params(C.Structure):
    _fields_ = [("theta", C.c_double), ("variants", C.c_uint), ("tau", C.c_double), ("sigma", C.c_double),
                ("cheb_degree", C.c_int), ("cheb_ratio", C.c_double), ("cheb_boost", C.c_double),
                ("power_iters", C.c_int),
                ("max_coarse", C.c_int), ("max_levels", C.c_int), ("pt_unit", C.c_int),
                ("onenorm_power", C.c_int), ("seed", C.c_uint64), ("lambda_override", C.c_double),
                ("max_iter", C.c_int), ("strength", C.c_int), ("krylov", C.c_int), ("restart", C.c_int),
                ("block_size", C.c_int), ("nullspace_dim", C.c_int)]


class Info(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("relres_true", C.c_double), ("levels", C.c_int),
                ("op_complexity", C.c_double)]


class _CSR(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rp", C.POINTER(C.c_int64)),
                ("ci", C.POINTER(C.c_int32)), ("v", C.POINTER(C.c_double))]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        vp = C.c_void_p
        L.oc_params_default.argtypes = [C.POINTER(Params)]
        L.oc_strength.argtypes = [C.c_int64, vp, vp, vp, C.c_double, vp]
        L.oc_filter.argtypes = [C.c_int64, vp, vp, vp, vp, C.c_int, C.c_double, C.POINTER(C.POINTER(_CSR)), vp]
        L.oc_mis2_aggregate.argtypes = [C.c_int64, vp, vp, vp, C.c_uint64, C.c_int, vp, vp]
        L.oc_mis2_aggregate.restype = C.c_int64
        L.oc_priority.argtypes = [C.c_uint64, C.c_int, C.c_int64]
        L.oc_priority.restype = C.c_uint64
        L.oc_sprsfy_mark.argtypes = [C.c_int64, vp, vp, vp, vp, vp, C.c_int64, vp]
        L.oc_constrain_row.argtypes = [C.c_int64, vp, C.c_int64, C.c_double]
        L.oc_spgemm.argtypes = [C.POINTER(_CSR), C.POINTER(_CSR), C.c_int64, C.POINTER(C.POINTER(_CSR))]
        L.oc_transpose.argtypes = [C.POINTER(_CSR), C.c_int64, C.POINTER(C.POINTER(_CSR))]
        L.oc_power_lambda.argtypes = [C.c_int64, vp, vp, vp, vp, C.c_int, C.c_uint64]
        L.oc_power_lambda.restype = C.c_double
        L.oc_power_stream_seed.argtypes = [C.c_uint64, C.c_int, C.c_int]
        L.oc_power_stream_seed.restype = C.c_uint64
        L.oc_cholesky.argtypes = [C.c_int64, vp, vp]
        L.oc_csr_free.argtypes = [C.POINTER(_CSR)]
        L.oc_setup.argtypes = [C.c_int64, vp, vp, vp, vp, C.POINTER(Params), C.POINTER(vp)]
        L.oc_setup_coords.argtypes = [C.c_int64, vp, vp, vp, vp, vp, C.c_int, C.POINTER(Params), C.POINTER(vp)]
        L.oc_distance_laplacian.argtypes = [C.c_int64, vp, vp, vp, C.c_int, vp]
        L.oc_coarse_coords.argtypes = [C.c_int64, vp, C.c_int64, vp, C.c_int, vp]
        L.oc_prolongator_only.argtypes = [C.c_int64, vp, vp, vp, vp, C.POINTER(Params), C.POINTER(vp)]
        L.oc_solve.argtypes = [vp, vp, vp, C.c_double, C.POINTER(Info)]
        L.oc_pcg_plain.argtypes = [C.c_int64, vp, vp, vp, vp, vp, C.c_double, C.c_int, C.POINTER(Info)]
        L.oc_gmres_plain.argtypes = [C.c_int64, vp, vp, vp, vp, vp, C.c_double, C.c_int, C.c_int, C.POINTER(Info)]
        L.oc_lu.argtypes = [C.c_int64, vp, vp]
        L.oc_lu_solve.argtypes = [C.c_int64, vp, vp, vp, vp]
        L.oc_vcycle.argtypes = [vp, vp, vp]
        L.oc_chebyshev_apply.argtypes = [C.c_int64, vp, vp, vp, vp, C.c_double, C.c_int, C.c_double, C.c_double,
                                         vp, vp]
        L.oc_free.argtypes = [vp]
        L.oc_nlevels.argtypes = [vp]
        L.oc_level_get.argtypes = [vp, C.c_int, C.c_int, vp, C.POINTER(C.c_int64)]
        L.oc_node_graph.argtypes = [C.c_int64, vp, vp, C.c_int, vp]
        L.oc_node_graph.restype = C.c_int64
        L.oc_node_fill.argtypes = [C.c_int64, vp, vp, vp, C.c_int, C.c_double, vp, vp, vp, vp, vp]
        L.oc_block_tentative.argtypes = [C.c_int64, C.c_int, C.c_int, vp, C.c_int64, vp, vp, vp]
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _arrs(A):
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.col, dtype=np.int32)
    v = np.ascontiguousarray(A.val, dtype=np.float64)
    return rp, ci, v


def _wrap(rp, ci, v, n):
    return _CSR(n, int(rp[-1]), rp.ctypes.data_as(C.POINTER(C.c_int64)), ci.ctypes.data_as(C.POINTER(C.c_int32)),
                v.ctypes.data_as(C.POINTER(C.c_double)))


def _take(cp):
    c = cp.contents
    n, nnz = c.n, c.nnz
    rp = np.ctypeslib.as_array(c.rp, shape=(n + 1,)).copy()
    ci = np.ctypeslib.as_array(c.ci, shape=(max(nnz, 1),))[:nnz].copy()
    v = np.ctypeslib.as_array(c.v, shape=(max(nnz, 1),))[:nnz].copy()
    lib().oc_csr_free(cp)
    return rp, ci, v


def params(**kw) -> Params:
    p = Params()
    lib().oc_params_default(C.byref(p))
    for k, val in kw.items():
        if k == "variants" and not isinstance(val, int):
            m = 0
            for s in val:
                m |= {"1norm": ONENORM, "offlmp": OFFLMP, "sprsfy": SPRSFY, "cnstrnt": CNSTRNT}[s.lower()]
            val = m
        setattr(p, k, val)
    return p


@dataclass
class SimpleCSR:
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self):
        return int(self.row_ptr[-1])

    def to_dense(self, ncol=None):
        ncol = self.n if ncol is None else ncol
        d = np.zeros((self.n, ncol))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        d[rows, self.col] = self.val
        return d


# ---------------------------------------------------------------- single steps

def strength(A, theta: float) -> np.ndarray:
    rp, ci, v = _arrs(A)
    out = np.zeros(len(ci), dtype=np.uint8)
    lib().oc_strength(A.n, _p(rp), _p(ci), _p(v), theta, _p(out))
    return out


def distance_laplacian(A, coords):
    """Values of the distance Laplacian on A's pattern (§3.1); (values, status)."""
    rp, ci, _ = _arrs(A)
    X = np.ascontiguousarray(coords, dtype=np.float64)
    dim = 1 if X.ndim == 1 else X.shape[1]
    out = np.zeros(max(len(ci), 1))
    st = lib().oc_distance_laplacian(A.n, _p(rp), _p(ci), _p(X), dim, _p(out))
    return out[:len(ci)], int(st)


def coarse_coords(agg, nagg: int, coords):
    a = np.ascontiguousarray(agg, dtype=np.int32)
    X = np.ascontiguousarray(coords, dtype=np.float64)
    dim = 1 if X.ndim == 1 else X.shape[1]
    out = np.zeros((max(nagg, 1), dim))
    st = lib().oc_coarse_coords(len(a), _p(a), nagg, _p(X), dim, _p(out))
    assert st == 0
    return out[:nagg]


def filtered(A, removed: np.ndarray, offlmp: bool = False, tau: float = 1.1):
    rp, ci, v = _arrs(A)
    rem = np.ascontiguousarray(removed, dtype=np.uint8)
    flag = np.zeros(max(A.n, 1), dtype=np.uint8)
    out = C.POINTER(_CSR)()
    st = lib().oc_filter(A.n, _p(rp), _p(ci), _p(v), _p(rem), int(offlmp), tau, C.byref(out), _p(flag))
    assert st == 0
    r, c, val = _take(out)
    return SimpleCSR(A.n, r, c, val), flag[:A.n]


def aggregate(A, strong: np.ndarray, seed: int = 0, level: int = 0):
    rp, ci, _ = _arrs(A)
    s = np.ascontiguousarray(strong, dtype=np.uint8)
    agg = np.zeros(max(A.n, 1), dtype=np.int32)
    root = np.zeros(max(A.n, 1), dtype=np.uint8)
    nagg = lib().oc_mis2_aggregate(A.n, _p(rp), _p(ci), _p(s), seed, level, _p(agg), _p(root))
    return agg[:A.n], root[:A.n], int(nagg)


def priority(seed: int, level: int, i: int) -> int:
    return int(lib().oc_priority(seed, level, i))


def sprsfy_mark(A, strong, agg, root, nagg, removed):
    rp, ci, _ = _arrs(A)
    rem = np.ascontiguousarray(removed, dtype=np.uint8).copy()
    npr = lib().oc_sprsfy_mark(A.n, _p(rp), _p(ci), _p(np.ascontiguousarray(strong, dtype=np.uint8)),
                               _p(np.ascontiguousarray(agg, dtype=np.int32)),
                               _p(np.ascontiguousarray(root, dtype=np.uint8)), nagg, _p(rem))
    return rem, int(npr)


def constrain_row(p, ptent_pos: int, ptent_val: float = 1.0):
    a = np.ascontiguousarray(p, dtype=np.float64).copy()
    code = lib().oc_constrain_row(len(a), _p(a), ptent_pos, ptent_val)
    return a, int(code)


def spgemm(A, B, ncolB: int) -> SimpleCSR:
    ra, ca, va = _arrs(A)
    rb, cb, vb = _arrs(B)
    wa, wb = _wrap(ra, ca, va, A.n), _wrap(rb, cb, vb, B.n)
    out = C.POINTER(_CSR)()
    st = lib().oc_spgemm(C.byref(wa), C.byref(wb), ncolB, C.byref(out))
    assert st == 0
    return SimpleCSR(A.n, *_take(out))


def transpose(A, ncol: int) -> SimpleCSR:
    ra, ca, va = _arrs(A)
    wa = _wrap(ra, ca, va, A.n)
    out = C.POINTER(_CSR)()
    st = lib().oc_transpose(C.byref(wa), ncol, C.byref(out))
    assert st == 0
    return SimpleCSR(ncol, *_take(out))


def power_lambda(A, D, sweeps: int, stream_seed: int) -> float:
    rp, ci, v = _arrs(A)
    d = np.ascontiguousarray(D, dtype=np.float64)
    return float(lib().oc_power_lambda(A.n, _p(rp), _p(ci), _p(v), _p(d), sweeps, stream_seed))


def power_stream_seed(seed: int, level: int, purpose: int) -> int:
    return int(lib().oc_power_stream_seed(seed, level, purpose))


def chebyshev_apply(A, lam: float, degree: int, x0=None, f=None, ratio: float = 10.0, boost: float = 1.1):
    """The V-cycle's smoother on its own: `degree` Chebyshev steps in D^-1 A on
    [boost*lam/ratio, boost*lam] applied to A x = f from x0 (zero if None); returns (x, status)."""
    rp, ci, v = _arrs(A)
    d = np.zeros(A.n)
    rows = np.repeat(np.arange(A.n), np.diff(rp))
    on = rows == ci
    d[rows[on]] = v[on]
    invd = 1.0 / d
    f = np.ascontiguousarray(f, dtype=np.float64)
    x = np.zeros(A.n) if x0 is None else np.ascontiguousarray(x0, dtype=np.float64).copy()
    st = lib().oc_chebyshev_apply(A.n, _p(rp), _p(ci), _p(v), _p(invd), lam, degree, ratio, boost, _p(f), _p(x))
    return x, int(st)


def cholesky(a: np.ndarray):
    a = np.ascontiguousarray(a, dtype=np.float64)
    n = a.shape[0]
    l = np.zeros_like(a)
    st = lib().oc_cholesky(n, _p(a), _p(l))
    return l, int(st)


def pcg_plain(A, b, tol: float, max_iter: int):
    rp, ci, v = _arrs(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(max(A.n, 1))
    info = Info()
    lib().oc_pcg_plain(A.n, _p(rp), _p(ci), _p(v), _p(b), _p(x), tol, max_iter, C.byref(info))
    return x[:A.n], info


def gmres_plain(A, b, tol: float, restart: int = 30, max_iter: int = 1000):
    rp, ci, v = _arrs(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(max(A.n, 1))
    info = Info()
    lib().oc_gmres_plain(A.n, _p(rp), _p(ci), _p(v), _p(b), _p(x), tol, restart, max_iter, C.byref(info))
    return x[:A.n], info


def lu_solve(a, b):
    """Dense LU with partial pivoting, then the solve: (x, status)."""
    a = np.ascontiguousarray(a, dtype=np.float64).copy()
    n = a.shape[0]
    piv = np.zeros(max(n, 1), dtype=np.int64)
    st = lib().oc_lu(n, _p(a), _p(piv))
    x = np.zeros(max(n, 1))
    if st == 0:
        lib().oc_lu_solve(n, _p(a), _p(piv), _p(np.ascontiguousarray(b, dtype=np.float64)), _p(x))
    return x[:n], int(st)


def node_strength(A, bs: int, theta: float):
    """Block strength of a system with bs unknowns per node: (node row pointer, node columns,
    block Frobenius norms, node strong flags, per-entry strong flags of A)."""
    rp, ci, v = _arrs(A)
    nn = A.n // bs
    nrp = np.zeros(nn + 1, dtype=np.int64)
    m = lib().oc_node_graph(A.n, _p(rp), _p(ci), bs, _p(nrp))
    assert m >= 0
    nci = np.zeros(max(m, 1), dtype=np.int32)
    nF = np.zeros(max(m, 1))
    ns = np.zeros(max(m, 1), dtype=np.uint8)
    strong = np.zeros(max(A.nnz, 1), dtype=np.uint8)
    st = lib().oc_node_fill(A.n, _p(rp), _p(ci), _p(v), bs, theta, _p(nrp), _p(nci), _p(nF), _p(ns), _p(strong))
    assert st == 0
    return nrp, nci[:m], nF[:m], ns[:m], strong[:A.nnz]


def block_tentative(n: int, bs: int, k: int, node_agg, nagg: int, B):
    """(Qv (n x k, row i = Pt's row i), Bc (k x nagg k), status) of the QR tentative prolongator."""
    node_agg = np.ascontiguousarray(node_agg, dtype=np.int32)
    B = np.ascontiguousarray(B, dtype=np.float64).reshape(-1)
    Qv = np.zeros(max(n * k, 1))
    Bc = np.zeros(max(nagg * k * k, 1))
    st = lib().oc_block_tentative(n, bs, k, _p(node_agg), nagg, _p(B), _p(Qv), _p(Bc))
    return Qv[:n * k].reshape(n, k), Bc[:nagg * k * k].reshape(k, nagg * k), int(st)


# ---------------------------------------------------------------- the whole method

_WHAT = {"A.rp": (0, np.int64), "A.ci": (1, np.int32), "A.v": (2, np.float64), "strong": (3, np.uint8),
         "removed": (4, np.uint8), "lumpflag": (5, np.uint8), "Abar.rp": (6, np.int64), "Abar.ci": (7, np.int32),
         "Abar.v": (8, np.float64), "agg": (9, np.int32), "root": (10, np.uint8), "P.rp": (11, np.int64),
         "P.ci": (12, np.int32), "P.v": (13, np.float64), "R.rp": (14, np.int64), "R.ci": (15, np.int32),
         "R.v": (16, np.float64), "Dsm": (17, np.float64), "scalars": (18, np.float64), "B": (19, np.float64),
         "cflag": (20, np.uint8), "chol": (21, np.float64), "coords": (22, np.float64), "bsk": (23, np.float64)}


class Hierarchy:
    """An oracle hierarchy; `level(l)` returns its arrays as numpy copies."""

    def __init__(self, handle, n):
        self._h = handle
        self.n = n

    def __del__(self):
        if getattr(self, "_h", None):
            lib().oc_free(self._h)
            self._h = None

    @property
    def nlevels(self) -> int:
        return int(lib().oc_nlevels(self._h))

    def get(self, level: int, what: str) -> np.ndarray:
        code, dt = _WHAT[what]
        ln = C.c_int64(0)
        st = lib().oc_level_get(self._h, level, code, None, C.byref(ln))
        assert st == 0
        out = np.zeros(max(ln.value, 1), dtype=dt)
        lib().oc_level_get(self._h, level, code, _p(out), C.byref(ln))
        return out[:ln.value]

    def level(self, l: int) -> dict:
        d = {k: self.get(l, k) for k in _WHAT}
        n = len(d["A.rp"]) - 1
        d["A"] = SimpleCSR(n, d["A.rp"], d["A.ci"], d["A.v"])
        if len(d["Abar.rp"]):
            d["Abar"] = SimpleCSR(n, d["Abar.rp"], d["Abar.ci"], d["Abar.v"])
            d["P"] = SimpleCSR(n, d["P.rp"], d["P.ci"], d["P.v"])
            d["R"] = SimpleCSR(len(d["R.rp"]) - 1, d["R.rp"], d["R.ci"], d["R.v"])
            sc = d["scalars"]
            d["lambda_bar"], d["omega"], d["lambda_cheb"], d["nagg"] = float(sc[0]), float(sc[1]), float(sc[2]), \
                int(sc[3])
        return d

    def solve(self, b, tol: float = 1e-8):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(max(self.n, 1))
        info = Info()
        st = lib().oc_solve(self._h, _p(b), _p(x), tol, C.byref(info))
        return x[:self.n], info, int(st)

    def vcycle(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        u = np.zeros(max(self.n, 1))
        lib().oc_vcycle(self._h, _p(f), _p(u))
        return u[:self.n]


def setup(A, nullspace=None, coords=None, **kw):
    """Returns (Hierarchy or None, status).  coords: (n, dim) coordinates of the rows, needed
    with strength=1 (distance-Laplacian strength, §3.1)."""
    rp, ci, v = _arrs(A)
    ns = None if nullspace is None else np.ascontiguousarray(nullspace, dtype=np.float64)
    p = params(**kw)
    h = C.c_void_p()
    if coords is not None:
        X = np.ascontiguousarray(coords, dtype=np.float64)
        dim = 1 if X.ndim == 1 else X.shape[1]
        st = lib().oc_setup_coords(A.n, _p(rp), _p(ci), _p(v), _p(ns), _p(X), dim, C.byref(p), C.byref(h))
    else:
        st = lib().oc_setup(A.n, _p(rp), _p(ci), _p(v), _p(ns), C.byref(p), C.byref(h))
    if st != 0:
        return None, int(st)
    return Hierarchy(h, A.n), 0


def prolongator_only(A, nullspace=None, **kw):
    rp, ci, v = _arrs(A)
    ns = None if nullspace is None else np.ascontiguousarray(nullspace, dtype=np.float64)
    p = params(**kw)
    h = C.c_void_p()
    st = lib().oc_prolongator_only(A.n, _p(rp), _p(ci), _p(v), _p(ns), C.byref(p), C.byref(h))
    if st != 0:
        return None, int(st)
    return Hierarchy(h, A.n), 0
