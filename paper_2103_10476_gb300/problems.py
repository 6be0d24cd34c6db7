"""Seeded synthetic inputs: Q1 (trilinear hexahedral) finite-element matrices and right-hand sides.

This module is the one place that both the CUDA path and the CPU oracle take their inputs
from.  It holds none of the SA-AMG arithmetic: it only assembles the linear system A u = f
of §1.1 Eq. (1) for the two operator families the paper studies (stretched meshes, §1.2 and
§3.2; large coefficient variation, §3.3) and draws right-hand sides.

Discretisation (the paper's §1.2 example and §3.1-§3.2 problems): axis-aligned tensor
mesh with per-axis element sizes, one diffusion coefficient c_e per element, Q1 elements
with exact (tensor-product) integration.  The element stiffness is
    c_e (Kx (x) My (x) Mz + Mx (x) Ky (x) Mz + Mx (x) My (x) Kz),
with the 1D stiffness K = [1, -1; -1, 1] / h and 1D mass M = h/6 [2, 1; 1, 2].
With Dirichlet boundaries the boundary nodes are eliminated (not stored); the unknowns are
the interior nodes, numbered i + Nx (j + Ny k).  The Neumann form keeps every node (its rows
sum to zero, so the constant is in the null space, §1.1).

Every structural neighbour of the 27-point stencil is stored, including entries whose
value cancels to zero (e.g. the face neighbours of a cube element); columns are sorted.
Values are exactly symmetric: entry (p, q) and (q, p) are summed over the same elements
in the same order.

Random numbers come from the SplitMix64 stream (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state s, output k (k = 1, 2, ...) is
mix(s + k * 0x9E3779B97F4A7C15) with the published 64-bit finaliser; a double in [0, 1)
is the top 53 bits times 2^-53.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_stream(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs start+1 .. start+n of the SplitMix64 stream with initial state `seed`."""
    k = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, n: int, start: int = 0) -> np.ndarray:
    """n doubles in [0, 1) from the SplitMix64 stream (top 53 bits * 2^-53)."""
    return (splitmix64_stream(seed, n, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def rhs_uniform(n: int, seed: int) -> np.ndarray:
    """Right-hand side with entries uniform in [-1, 1), in unknown-index order."""
    return 2.0 * uniform01(seed, n) - 1.0


@dataclass
class CSR:
    """Square CSR matrix: int64 row pointer, int32 sorted columns, float64 values."""
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        d[rows, self.col] = self.val
        return d


def _axis_options(h: np.ndarray, dirichlet: bool):
    """Per axis: for each unknown node index and offset d in {-1, 0, 1}, the (up to two)
    elements shared by the node and its neighbour, with 1D stiffness and mass factors.

    Returns (n_nodes, opts) where opts[d] is a list of two slots, each a tuple of arrays
    (valid, element, K, M) over the node index; slots are in ascending element order.
    """
    ne = len(h)
    if dirichlet:
        nn = ne - 1
        full = np.arange(1, ne)          # full-mesh index of interior node i
    else:
        nn = ne + 1
        full = np.arange(0, ne + 1)
    opts = {}
    for d in (-1, 0, 1):
        slots = []
        cands = [full - 1, full] if d == 0 else ([full - 1] if d == -1 else [full])
        for e in cands:
            nb = full + d
            valid = (e >= 0) & (e < ne)
            if dirichlet:
                valid &= (nb >= 1) & (nb <= ne - 1)
            else:
                valid &= (nb >= 0) & (nb <= ne)
            ec = np.clip(e, 0, ne - 1)
            he = h[ec]
            if d == 0:
                K = 1.0 / he
                M = 2.0 * he / 6.0
            else:
                K = -1.0 / he
                M = he / 6.0
            slots.append((valid, ec, K, M))
        opts[d] = slots
    return nn, opts


_GEN = None


def _gen_lib():
    """The C assembly of q1gen.c (built on first use)."""
    global _GEN
    if _GEN is None:
        import ctypes as C
        from . import build as _build
        L = C.CDLL(_build.build_generator())
        L.q1_assemble.restype = C.c_int64
        L.q1_assemble.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
        _GEN = L
    return _GEN


def _q1_matrix_c(hx, hy, hz, coef, dirichlet: bool) -> CSR:
    L = _gen_lib()
    nex, ney, nez = len(hx), len(hy), len(hz)
    nx, ny, nz = ((nex - 1, ney - 1, nez - 1) if dirichlet else (nex + 1, ney + 1, nez + 1))
    n = max(nx, 0) * max(ny, 0) * max(nz, 0)
    rp = np.zeros(n + 1, dtype=np.int64)
    col = np.empty(27 * n, dtype=np.int32)
    val = np.empty(27 * n, dtype=np.float64)
    c = None if coef is None else np.ascontiguousarray(coef, dtype=np.float64)
    nnz = L.q1_assemble(nex, ney, nez, hx.ctypes.data, hy.ctypes.data, hz.ctypes.data,
                        None if c is None else c.ctypes.data, int(dirichlet), rp.ctypes.data, col.ctypes.data,
                        val.ctypes.data)
    if nnz < 0:
        raise MemoryError("q1_assemble")
    return CSR(n, rp, col[:nnz], val[:nnz], meta={"grid": (nx, ny, nz)})


def q1_matrix(hx, hy, hz, coef=None, dirichlet: bool = True, engine: str = "numpy") -> CSR:
    """Assemble the Q1 finite-element diffusion matrix on a tensor mesh.

    engine "c" runs the same assembly (the same operations in the same order, so the same
    bits) in q1gen.c, for large operators.

    hx, hy, hz: element sizes along each axis (lengths nex, ney, nez).
    coef: per-element coefficient, shape (nez, ney, nex) (element order
          e = ex + nex (ey + ney ez)), or None for 1.
    """
    hx = np.ascontiguousarray(hx, dtype=np.float64)
    hy = np.ascontiguousarray(hy, dtype=np.float64)
    hz = np.ascontiguousarray(hz, dtype=np.float64)
    if engine == "c":
        return _q1_matrix_c(hx, hy, hz, coef, dirichlet)
    nx, ox = _axis_options(hx, dirichlet)
    ny, oy = _axis_options(hy, dirichlet)
    nz, oz = _axis_options(hz, dirichlet)
    if coef is None:
        coef = np.ones((len(hz), len(hy), len(hx)))
    coef = np.asarray(coef, dtype=np.float64)
    n = nx * ny * nz
    vals = np.zeros((27, nz, ny, nx))
    mask = np.zeros((27, nz, ny, nx), dtype=bool)
    t = 0
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                acc = np.zeros((nz, ny, nx))
                any_valid = np.zeros((nz, ny, nx), dtype=bool)
                for (vz, ez, Kz, Mz) in oz[dz]:
                    for (vy, ey, Ky, My) in oy[dy]:
                        for (vx, ex, Kx, Mx) in ox[dx]:
                            v = vz[:, None, None] & vy[None, :, None] & vx[None, None, :]
                            c = coef[ez[:, None, None], ey[None, :, None], ex[None, None, :]]
                            KZ, MZ = Kz[:, None, None], Mz[:, None, None]
                            KY, MY = Ky[None, :, None], My[None, :, None]
                            KX, MX = Kx[None, None, :], Mx[None, None, :]
                            term = (KX * MY) * MZ + (MX * KY) * MZ + (MX * MY) * KZ
                            acc = acc + np.where(v, c * term, 0.0)
                            any_valid |= v
                vals[t] = acc
                mask[t] = any_valid
                t += 1
    # row-major (k, j, i) with the 27 offsets innermost, already in ascending column order
    vals = np.moveaxis(vals, 0, -1).reshape(n, 27)
    mask = np.moveaxis(mask, 0, -1).reshape(n, 27)
    offs = np.array([dx + nx * (dy + ny * dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)],
                    dtype=np.int64)
    cols = np.arange(n, dtype=np.int64)[:, None] + offs[None, :]
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = cols[mask].astype(np.int32)
    val = vals[mask]
    return CSR(n, row_ptr, col, np.ascontiguousarray(val), meta={"grid": (nx, ny, nz)})


# ----------------------------------------------------------------------------------------
# The problem families used as workloads (synthetic stand-ins for the paper's meshes).
# ----------------------------------------------------------------------------------------

def laplace_cube(N: int) -> CSR:
    """Unit cube, N^3 interior nodes, coefficient 1, homogeneous Dirichlet (h = 1/(N+1))."""
    h = np.full(N + 1, 1.0 / (N + 1))
    A = q1_matrix(h, h, h)
    A.meta.update(family="laplace_cube", N=N)
    return A


def stretched_box(N: int, ratio: float = 1.1, engine: str = "numpy") -> CSR:
    """N^3 interior nodes; unit spacing in x and y, z element layers h_z(k) = ratio^k,
    k = 0..N (the stretched-mesh setting of §1.2 and §3.2: aspect ratios 1 to ratio^N)."""
    hxy = np.ones(N + 1)
    hz = ratio ** np.arange(N + 1, dtype=np.float64)
    A = q1_matrix(hxy, hxy, hz, engine=engine)
    A.meta.update(family="stretched_box", N=N, ratio=ratio)
    return A


def random_coefficient_cube(N: int, seed: int, decades: float = 3.0, engine: str = "numpy") -> CSR:
    """Unit cube, N^3 interior nodes, per-element coefficient 10^(2*decades*u - decades),
    u ~ U[0, 1) from SplitMix64(seed) in element order (the coefficient-variation setting
    of §3.3)."""
    ne = N + 1
    u = uniform01(seed, ne ** 3).reshape(ne, ne, ne)
    coef = 10.0 ** (2.0 * decades * u - decades)
    h = np.full(ne, 1.0 / ne)
    A = q1_matrix(h, h, h, coef, engine=engine)
    A.meta.update(family="random_coefficient_cube", N=N, seed=seed, decades=decades)
    return A


def neumann_box(nx: int, ny: int, nz: int, hx=1.0, hy=1.0, hz=1.0, coef=None) -> CSR:
    """Pure-Neumann Q1 matrix on nx*ny*nz nodes (all nodes kept; rows sum to zero)."""
    A = q1_matrix(np.full(nx - 1, hx), np.full(ny - 1, hy), np.full(nz - 1, hz), coef, dirichlet=False)
    A.meta.update(family="neumann_box")
    return A


# ----------------------------------------------------------------------------------------
# Named workloads (sizes and seeds of the five benchmark configurations).
# ----------------------------------------------------------------------------------------

VARIANT_BITS = {"1norm": 1, "offlmp": 2, "sprsfy": 4, "cnstrnt": 8}


def variants_mask(names) -> int:
    m = 0
    for s in names:
        m |= VARIANT_BITS[s.lower()]
    return m


def workload_laplace20():
    """27-point Q1 Laplacian, unit cube, 20^3 interior nodes; theta = 0; RHS seed 0."""
    A = laplace_cube(20)
    return A, rhs_uniform(A.n, 0), dict(theta=0.0, variants=0)


def workload_stretched64(N: int = 64):
    """Stretched box, 64^3 interior nodes, z ratio 1.1; theta = 0.02; RHS seed 1."""
    A = stretched_box(N, 1.1)
    return A, rhs_uniform(A.n, 1), dict(theta=0.02)


def workload_randcoef128(N: int = 128):
    """Random-coefficient cube, 128^3 interior nodes, 10^U(-3,3) with seed 2; theta = 0.02,
    1Norm + OffLmp; RHS seed 2."""
    A = random_coefficient_cube(N, 2, 3.0)
    return A, rhs_uniform(A.n, 2), dict(theta=0.02, variants=VARIANT_BITS["1norm"] | VARIANT_BITS["offlmp"])


def batched_systems(count: int = 512, seed: int = 3, nmin: int = 8, nmax: int = 40, engine: str = "numpy"):
    """`count` independent systems with edge N ~ U{nmin..nmax}; the first half stretched
    (z ratio ~ U[1.05, 1.2]), the second half coefficient 10^U(-2,2).  System s draws from
    the SplitMix64 stream seed ^ (s+1) << 32."""
    out = []
    for s in range(count):
        sub = seed ^ ((s + 1) << 32)
        u = uniform01(sub, 3)
        N = nmin + int(u[0] * (nmax - nmin + 1))
        if s < count // 2:
            ratio = 1.05 + 0.15 * float(u[1])
            A = stretched_box(N, ratio, engine=engine)
        else:
            A = random_coefficient_cube(N, sub ^ 0xC0EF, 2.0, engine=engine)
        out.append((A, rhs_uniform(A.n, sub ^ 0xB)))
    return out


def serving_stream(duration_s: float = 60.0, rate: float = 200.0, seed: int = 4, nmin: int = 16, nmax: int = 96,
                   repeat: float = 0.3, rhs_max: int = 8):
    """A request stream for the server: Poisson arrivals at `rate` per second over
    `duration_s`; each request after the first repeats an earlier operator (uniformly among
    those seen) with probability `repeat`, otherwise it brings a new one: edge N log-uniform
    in [nmin, nmax] nodes, half stretched boxes (z ratio U[1.05, 1.2]), half
    random-coefficient cubes (10^U(-2, 2)); 1..rhs_max right-hand sides.  Request r draws
    six uniforms from SplitMix64(seed) at offset 6 r.

    Returns (requests, operators): requests are tuples (arrival_s, operator index, nrhs,
    rhs seed); operators are tuples (family, N, parameter) for make_operator."""
    reqs, ops = [], []
    t = 0.0
    r = 0
    while True:
        u = uniform01(seed, 6, start=6 * r)
        t += -np.log1p(-float(u[0])) / rate
        if t >= duration_s:
            break
        if ops and float(u[1]) < repeat:
            k = min(int(float(u[2]) * len(ops)), len(ops) - 1)
        else:
            N = int(np.floor(nmin * (nmax / nmin) ** float(u[3])))
            N = min(max(N, nmin), nmax)
            if float(u[4]) < 0.5:
                ops.append(("stretched", N, 1.05 + 0.15 * float(u[2])))
            else:
                ops.append(("randcoef", N, (seed << 40) ^ (len(ops) + 1)))
            k = len(ops) - 1
        nrhs = 1 + min(int(float(u[5]) * rhs_max), rhs_max - 1)
        reqs.append((t, k, nrhs, (seed << 48) ^ (r + 1)))
        r += 1
    return reqs, ops


def make_operator(op, engine: str = "c") -> CSR:
    """The matrix of one serving_stream operator."""
    family, N, param = op
    if family == "stretched":
        return stretched_box(N, param, engine=engine)
    return random_coefficient_cube(N, param, 2.0, engine=engine)


def dirichlet_stencil_row(A: CSR, i: int, j: int, k: int) -> dict:
    """The 27-point row of interior node (i, j, k), keyed by offset (dx, dy, dz)."""
    nx, ny, nz = A.meta["grid"]
    r = i + nx * (j + ny * k)
    out = {}
    for e in range(int(A.row_ptr[r]), int(A.row_ptr[r + 1])):
        c = int(A.col[e])
        dz, rem = divmod(c, nx * ny)
        dy, dx = divmod(rem, nx)
        out[(dx - i, dy - j, dz - k)] = float(A.val[e])
    return out


__all__ = [
    "CSR", "splitmix64_stream", "uniform01", "rhs_uniform", "q1_matrix", "laplace_cube",
    "stretched_box", "random_coefficient_cube", "neumann_box", "workload_laplace20",
    "workload_stretched64", "workload_randcoef128", "batched_systems", "serving_stream", "make_operator",
    "VARIANT_BITS",
    "variants_mask", "dirichlet_stencil_row",
]
