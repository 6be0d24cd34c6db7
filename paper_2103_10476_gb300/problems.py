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


# ------------------------------------------------------------------------------ general hexahedra
# Q1 elements on a structured grid of arbitrary (non-inverted) trilinear hexahedra, for the
# distance-Laplacian experiments of §3.1-§3.2 (a randomly perturbed cube and a triaxially
# graded cube with a reaction term).  Element (i, j, k) has the 8 nodes (i + ax, j + ay,
# k + az), a in {0,1}^3, local number ax + 2 ay + 4 az, reference coordinates 2a - 1.  Its
# matrix is c_e * stiffness + r_e * mass, integrated with the 2 x 2 x 2 Gauss rule (points
# +-1/sqrt(3), weights 1), which is exact for the mass and stiffness of axis-aligned boxes.
# Entry (p, q) of the global matrix adds its element contributions in increasing element
# number (e = i + nex (j + ney k)); each element's matrix is exactly symmetric, so the global
# matrix is too.

_GAUSS = 1.0 / np.sqrt(3.0)


def _hex_element_matrices(Xe: np.ndarray, coef: np.ndarray, reaction: np.ndarray | None,
                          velocity=None) -> np.ndarray:
    """Xe: (E, 8, 3) node coordinates; coef, reaction: (E,); velocity: constant 3-vector of the
    convection term sum over Gauss points of N_a (v . grad N_b) (nonsymmetric), or None.
    Returns (E, 8, 8)."""
    E = Xe.shape[0]
    vel = None if velocity is None else np.asarray(velocity, dtype=np.float64)
    sgn = np.array([[2 * (a & 1) - 1, 2 * ((a >> 1) & 1) - 1, 2 * ((a >> 2) & 1) - 1] for a in range(8)],
                   dtype=np.float64)
    K = np.zeros((E, 8, 8))
    M = np.zeros((E, 8, 8)) if reaction is not None else None
    for gz in (-_GAUSS, _GAUSS):
        for gy in (-_GAUSS, _GAUSS):
            for gx in (-_GAUSS, _GAUSS):
                g = np.array([gx, gy, gz])
                f = 1.0 + sgn * g                       # (8, 3): 1 + xi_a xi per axis
                N = f[:, 0] * f[:, 1] * f[:, 2] / 8.0   # shape functions
                dN = np.empty((8, 3))                   # d N_a / d xi_q
                dN[:, 0] = sgn[:, 0] * f[:, 1] * f[:, 2] / 8.0
                dN[:, 1] = f[:, 0] * sgn[:, 1] * f[:, 2] / 8.0
                dN[:, 2] = f[:, 0] * f[:, 1] * sgn[:, 2] / 8.0
                # J[e, p, q] = sum_a X[e, a, p] dN[a, q]
                J = np.zeros((E, 3, 3))
                for a in range(8):
                    J += Xe[:, a, :, None] * dN[a][None, None, :]
                c00 = J[:, 1, 1] * J[:, 2, 2] - J[:, 1, 2] * J[:, 2, 1]
                c01 = J[:, 1, 2] * J[:, 2, 0] - J[:, 1, 0] * J[:, 2, 2]
                c02 = J[:, 1, 0] * J[:, 2, 1] - J[:, 1, 1] * J[:, 2, 0]
                det = J[:, 0, 0] * c00 + J[:, 0, 1] * c01 + J[:, 0, 2] * c02
                if np.any(det <= 0.0):
                    raise ValueError("inverted or degenerate hexahedron")
                inv = np.empty((E, 3, 3))           # inv = J^-1 (adjugate / det)
                inv[:, 0, 0] = c00
                inv[:, 1, 0] = c01
                inv[:, 2, 0] = c02
                inv[:, 0, 1] = J[:, 0, 2] * J[:, 2, 1] - J[:, 0, 1] * J[:, 2, 2]
                inv[:, 1, 1] = J[:, 0, 0] * J[:, 2, 2] - J[:, 0, 2] * J[:, 2, 0]
                inv[:, 2, 1] = J[:, 0, 1] * J[:, 2, 0] - J[:, 0, 0] * J[:, 2, 1]
                inv[:, 0, 2] = J[:, 0, 1] * J[:, 1, 2] - J[:, 0, 2] * J[:, 1, 1]
                inv[:, 1, 2] = J[:, 0, 2] * J[:, 1, 0] - J[:, 0, 0] * J[:, 1, 2]
                inv[:, 2, 2] = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
                inv /= det[:, None, None]
                # physical gradients G[e, a, p] = sum_q dN[a, q] inv[e, q, p]
                G = np.zeros((E, 8, 3))
                for q in range(3):
                    G += dN[None, :, q, None] * inv[:, None, q, :]
                w = (det * coef)[:, None, None]
                K += w * (G[:, :, None, 0] * G[:, None, :, 0] + G[:, :, None, 1] * G[:, None, :, 1]
                          + G[:, :, None, 2] * G[:, None, :, 2])
                if M is not None:
                    M += (det * reaction)[:, None, None] * (N[:, None] * N[None, :])[None]
                if vel is not None:
                    vg = G[:, :, 0] * vel[0] + G[:, :, 1] * vel[1] + G[:, :, 2] * vel[2]    # (E, 8): v . grad N_b
                    K += det[:, None, None] * (N[None, :, None] * vg[:, None, :])
    return K if M is None else K + M


def hex_q1_matrix(X: np.ndarray, Y: np.ndarray, Z: np.ndarray, coef=None, reaction=None,
                  dirichlet: bool = True, velocity=None) -> CSR:
    """Q1 matrix of the structured hexahedral grid with node coordinates X, Y, Z (each of
    shape (nez + 1, ney + 1, nex + 1), node (i, j, k) at [k, j, i]).  coef: per-element
    diffusion (shape (nez, ney, nex) or None for 1); reaction: per-element coefficient of the
    mass term (the 1/sigma of §3.2's reaction-diffusion equation) or None.  With Dirichlet
    boundaries the boundary nodes are eliminated.  meta["coords"] holds the (n, 3)
    coordinates of the unknowns, in unknown order."""
    X, Y, Z = (np.ascontiguousarray(a, dtype=np.float64) for a in (X, Y, Z))
    nz1, ny1, nx1 = X.shape
    nex, ney, nez = nx1 - 1, ny1 - 1, nz1 - 1
    E = nex * ney * nez
    ei, ej, ek = np.meshgrid(np.arange(nex), np.arange(ney), np.arange(nez), indexing="xy")
    # element order e = i + nex (j + ney k)
    ei = np.transpose(ei, (2, 0, 1)).ravel()
    ej = np.transpose(ej, (2, 0, 1)).ravel()
    ek = np.transpose(ek, (2, 0, 1)).ravel()
    nodes = np.empty((E, 8), dtype=np.int64)
    Xe = np.empty((E, 8, 3))
    for a in range(8):
        ii, jj, kk = ei + (a & 1), ej + ((a >> 1) & 1), ek + ((a >> 2) & 1)
        nodes[:, a] = ii + nx1 * (jj + ny1 * kk)
        Xe[:, a, 0] = X[kk, jj, ii]
        Xe[:, a, 1] = Y[kk, jj, ii]
        Xe[:, a, 2] = Z[kk, jj, ii]
    c = np.ones(E) if coef is None else np.asarray(coef, dtype=np.float64).reshape(nez, ney, nex).ravel()
    r = None if reaction is None else np.broadcast_to(np.asarray(reaction, dtype=np.float64),
                                                      (nez, ney, nex)).ravel()
    Ke = _hex_element_matrices(Xe, c, r, velocity)
    # unknown numbering
    if dirichlet:
        inner = np.zeros((nz1, ny1, nx1), dtype=bool)
        inner[1:-1, 1:-1, 1:-1] = True
    else:
        inner = np.ones((nz1, ny1, nx1), dtype=bool)
    inner = inner.ravel()
    num = np.full(inner.size, -1, dtype=np.int64)
    num[inner] = np.arange(int(inner.sum()))
    n = int(inner.sum())
    rows = np.repeat(num[nodes], 8, axis=1).ravel()          # (E, 64): row of entry (a, b)
    cols = np.tile(num[nodes], (1, 8)).ravel()
    vals = Ke.reshape(E, 64).ravel()
    keep = (rows >= 0) & (cols >= 0)
    rows, cols, vals = rows[keep], cols[keep], vals[keep]
    elem = np.repeat(np.arange(E), 64)[keep]
    order = np.lexsort((elem, cols, rows))                    # by row, column, element
    rows, cols, vals = rows[order], cols[order], vals[order]
    key = rows * n + cols
    start = np.flatnonzero(np.r_[True, key[1:] != key[:-1]])
    cnt = np.diff(np.r_[start, key.size])
    acc = vals[start].copy()
    for k in range(1, int(cnt.max()) if cnt.size else 1):   # contributions in element order
        m = cnt > k
        acc[m] = acc[m] + vals[start[m] + k]
    urow = rows[start]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, urow + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    coords = np.stack([X.ravel()[inner], Y.ravel()[inner], Z.ravel()[inner]], axis=1)
    return CSR(n, row_ptr, cols[start].astype(np.int32), acc,
               meta={"grid": (nx1 - 2, ny1 - 2, nz1 - 2) if dirichlet else (nx1, ny1, nz1), "coords": coords})


def _hex_elasticity_matrices(Xe: np.ndarray, lam: float, mu: float) -> np.ndarray:
    """Xe: (E, 8, 3) node coordinates.  Isotropic linear elasticity with Lame parameters lam,
    mu on trilinear hexahedra, 2x2x2 Gauss rule: entry (3a + p, 3b + q) of the (E, 24, 24)
    element matrices is the sum over Gauss points of
    det J (lam G_ap G_bq + mu G_aq G_bp + mu delta_pq grad N_a . grad N_b)."""
    E = Xe.shape[0]
    sgn = np.array([[2 * (a & 1) - 1, 2 * ((a >> 1) & 1) - 1, 2 * ((a >> 2) & 1) - 1] for a in range(8)],
                   dtype=np.float64)
    K = np.zeros((E, 8, 3, 8, 3))
    for gz in (-_GAUSS, _GAUSS):
        for gy in (-_GAUSS, _GAUSS):
            for gx in (-_GAUSS, _GAUSS):
                g = np.array([gx, gy, gz])
                f = 1.0 + sgn * g
                dN = np.empty((8, 3))
                dN[:, 0] = sgn[:, 0] * f[:, 1] * f[:, 2] / 8.0
                dN[:, 1] = f[:, 0] * sgn[:, 1] * f[:, 2] / 8.0
                dN[:, 2] = f[:, 0] * f[:, 1] * sgn[:, 2] / 8.0
                J = np.einsum("eap,aq->epq", Xe, dN)
                det = np.linalg.det(J)
                if np.any(det <= 0.0):
                    raise ValueError("inverted or degenerate hexahedron")
                inv = np.linalg.inv(J)
                G = np.einsum("aq,eqp->eap", dN, inv)             # physical gradients
                w = det[:, None, None, None, None]
                lap = np.einsum("eap,ebp->eab", G, G)
                K += w * (lam * np.einsum("eap,ebq->eapbq", G, G) + mu * np.einsum("eaq,ebp->eapbq", G, G)
                          + mu * lap[:, :, None, :, None] * np.eye(3)[None, None, :, None, :])
    return K.reshape(E, 24, 24)


def elasticity_box(hx, hy, hz, E: float = 1.0, nu: float = 0.3, clamp: bool = True) -> CSR:
    """3D linear elasticity on the tensor mesh with element sizes hx, hy, hz (Q1 hexahedra,
    2x2x2 Gauss rule), three unknowns per node interleaved (unknown 3 v + c is displacement
    component c of node v).  clamp: the nodes of the face x = 0 are fixed (eliminated), making
    the operator positive definite; otherwise every node is kept (the six rigid-body motions
    span the kernel).  meta: "coords" (per node), "block_size" 3, "rbm" (n x 6, column-major
    as 6 vectors of length n: translations x, y, z, then rotations about the z, x and y axes
    through the centroid of the kept nodes)."""
    hx, hy, hz = (np.asarray(h, dtype=np.float64) for h in (hx, hy, hz))
    ax = [np.r_[0.0, np.cumsum(h)] for h in (hx, hy, hz)]
    nx1, ny1, nz1 = (len(a) for a in ax)
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    nex, ney, nez = nx1 - 1, ny1 - 1, nz1 - 1
    ne = nex * ney * nez
    ei, ej, ek = np.meshgrid(np.arange(nex), np.arange(ney), np.arange(nez), indexing="xy")
    ei = np.transpose(ei, (2, 0, 1)).ravel()
    ej = np.transpose(ej, (2, 0, 1)).ravel()
    ek = np.transpose(ek, (2, 0, 1)).ravel()
    nodes = np.empty((ne, 8), dtype=np.int64)
    Xe = np.empty((ne, 8, 3))
    for a in range(8):
        ii, jj, kk = ei + (a & 1), ej + ((a >> 1) & 1), ek + ((a >> 2) & 1)
        nodes[:, a] = ii + nx1 * (jj + ny1 * kk)
        Xe[:, a, 0] = X[kk, jj, ii]
        Xe[:, a, 1] = Y[kk, jj, ii]
        Xe[:, a, 2] = Z[kk, jj, ii]
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    Ke = _hex_elasticity_matrices(Xe, lam, mu)
    keep_node = np.ones((nz1, ny1, nx1), dtype=bool)
    if clamp:
        keep_node[:, :, 0] = False
    keep_node = keep_node.ravel()
    num = np.full(keep_node.size, -1, dtype=np.int64)
    num[keep_node] = np.arange(int(keep_node.sum()))
    nn = int(keep_node.sum())
    n = 3 * nn
    dof = np.where(num[nodes][:, :, None] >= 0, 3 * num[nodes][:, :, None] + np.arange(3)[None, None, :], -1)
    dof = dof.reshape(ne, 24)
    rows = np.repeat(dof, 24, axis=1).ravel()
    cols = np.tile(dof, (1, 24)).ravel()
    vals = Ke.reshape(ne, 576).ravel()
    keep = (rows >= 0) & (cols >= 0)
    rows, cols, vals = rows[keep], cols[keep], vals[keep]
    elem = np.repeat(np.arange(ne), 576)[keep]
    order = np.lexsort((elem, cols, rows))                    # by row, column, element
    rows, cols, vals = rows[order], cols[order], vals[order]
    key = rows * n + cols
    start = np.flatnonzero(np.r_[True, key[1:] != key[:-1]])
    cnt = np.diff(np.r_[start, key.size])
    acc = vals[start].copy()
    for k in range(1, int(cnt.max()) if cnt.size else 1):   # contributions in element order
        m = cnt > k
        acc[m] = acc[m] + vals[start[m] + k]
    urow = rows[start]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, urow + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    coords = np.stack([X.ravel()[keep_node], Y.ravel()[keep_node], Z.ravel()[keep_node]], axis=1)
    return CSR(n, row_ptr, cols[start].astype(np.int32), acc,
               meta={"coords": coords, "block_size": 3, "rbm": rigid_body_modes(coords),
                     "grid": (nx1, ny1, nz1), "family": "elasticity", "E": E, "nu": nu, "clamp": clamp})


def rigid_body_modes(coords: np.ndarray) -> np.ndarray:
    """The six rigid-body motions of nodes at coords (nn x 3) as 6 vectors of length 3 nn,
    stored one after another (unknown 3 v + c = component c of node v): translations along
    x, y, z, then rotations about the z, x and y axes through the centroid."""
    nn = coords.shape[0]
    c = coords - coords.mean(axis=0)
    x, y, z = c[:, 0], c[:, 1], c[:, 2]
    B = np.zeros((6, nn, 3))
    for t in range(3):
        B[t, :, t] = 1.0
    B[3, :, 0], B[3, :, 1] = -y, x          # about z
    B[4, :, 1], B[4, :, 2] = -z, y          # about x
    B[5, :, 0], B[5, :, 2] = z, -x          # about y
    return np.ascontiguousarray(B.reshape(6, 3 * nn))


def workload_elasticity(N: int = 40):
    """Cantilever-like elasticity block: N^3 unit elements, E = 1, nu = 0.3, face x = 0 clamped
    (N (N+1)^2 nodes, three unknowns each); near-null space = the six rigid-body modes;
    theta = 0.02, traditional SA; RHS seed 6."""
    h = np.ones(N)
    A = elasticity_box(h, h, h)
    return A, rhs_uniform(A.n, 6), dict(theta=0.02, variants=0, block_size=3, nullspace_dim=6)


def perturbed_cube(ne: int = 60, seed: int = 5, amplitude: float = 0.2, zscale: float = 100.0) -> CSR:
    """§3.1's randomly perturbed cube: the Laplacian on [0,1] x [0,1] x [0,zscale] with ne
    elements per direction; every node of the uniform grid moves along each axis by
    amplitude * u / ne (u uniform in [0, 1), SplitMix64 stream `seed`, three draws per node
    in node order x, y, z) before z is scaled by zscale, so the z spacing is zscale times
    the x and y spacing and the hexahedra are general trilinear ones."""
    n1 = ne + 1
    u = uniform01(seed, 3 * n1 ** 3).reshape(n1, n1, n1, 3)   # [k, j, i, axis]
    g = np.arange(n1, dtype=np.float64) / ne
    Z0, Y0, X0 = np.meshgrid(g, g, g, indexing="ij")
    X = X0 + amplitude * u[..., 0] / ne
    Y = Y0 + amplitude * u[..., 1] / ne
    Z = (Z0 + amplitude * u[..., 2] / ne) * zscale
    A = hex_q1_matrix(X, Y, Z)
    A.meta.update(family="perturbed", ne=ne, seed=seed)
    return A


def graded_sizes(k: float, ne: int = 60) -> np.ndarray:
    """Element sizes varying linearly from 0.1 to k/10 over ne elements (length 3(k+1)
    for ne = 60), the grading of §3.2's triaxially stretched cube."""
    return 0.1 + (k / 10.0 - 0.1) * np.arange(ne, dtype=np.float64) / (ne - 1)


def graded_cube(kx: float, ky: float, kz: float, sigma: float, ne: int = 60) -> CSR:
    """§3.2's triaxially stretched cube: sigma^-1 u - Laplace(u) on the tensor mesh with
    graded_sizes(kx), (ky), (kz) along x, y, z (positive row sums from the reaction term)."""
    ax = [np.r_[0.0, np.cumsum(graded_sizes(k, ne))] for k in (kx, ky, kz)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    A = hex_q1_matrix(X, Y, Z, reaction=1.0 / sigma)
    A.meta.update(family="graded", k=(kx, ky, kz), sigma=sigma, ne=ne)
    return A


def convection_diffusion_box(N: int, velocity=(1.0, 0.5, 0.25), ratio: float = 1.1) -> CSR:
    """A nonsymmetric stand-in (§3's wind pressure system is solved by GMRES): -Laplace(u) +
    v . grad(u) with constant velocity v, Galerkin Q1 on the stretched box of `stretched_box`
    (unit x and y spacing, z spacing ratio^k), N^3 interior nodes, Dirichlet boundaries.  The
    element Peclet number |v| h / 2 is below 1 on the unit-spaced axes."""
    ax = np.arange(N + 2, dtype=np.float64)
    az = np.r_[0.0, np.cumsum(ratio ** np.arange(N + 1, dtype=np.float64))]
    Z, Y, X = np.meshgrid(az, ax, ax, indexing="ij")
    A = hex_q1_matrix(X, Y, Z, velocity=velocity)
    A.meta.update(family="convection", velocity=tuple(velocity), ratio=ratio)
    return A


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


def workload_convdiff64(N: int = 64):
    """Nonsymmetric stand-in for §3's pressure system (solved there by GMRES with SA):
    convection-diffusion with velocity (0.16, 0.08, 0.04) on the box with unit x and y spacing
    and z ratio 1.05, 64^3 interior nodes (cell Peclet numbers |v_i| h_i / 2 below 0.5); theta = 0.02,
    1Norm + OffLmp, GMRES(30); RHS seed 1."""
    A = convection_diffusion_box(N, velocity=(0.16, 0.08, 0.04), ratio=1.05)
    return A, rhs_uniform(A.n, 1), dict(theta=0.02, variants=VARIANT_BITS["1norm"] | VARIANT_BITS["offlmp"],
                                        krylov=1, restart=30)


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
    "variants_mask", "dirichlet_stencil_row", "hex_q1_matrix", "perturbed_cube", "graded_sizes",
    "graded_cube", "convection_diffusion_box", "workload_convdiff64", "elasticity_box", "rigid_body_modes",
    "workload_elasticity",
]
