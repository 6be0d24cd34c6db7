"""Small test matrices built by hand (no SA-AMG arithmetic)."""
import numpy as np

from paper_2103_10476_gb300.problems import CSR


def csr_from_dense(d: np.ndarray, keep_zeros_pattern: np.ndarray | None = None) -> CSR:
    """CSR of a dense matrix; entries where d != 0 (or where keep_zeros_pattern is True) are stored."""
    d = np.asarray(d, dtype=np.float64)
    n = d.shape[0]
    pat = (d != 0) if keep_zeros_pattern is None else (keep_zeros_pattern | (d != 0))
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum(pat.sum(1))
    rows, cols = np.nonzero(pat)
    return CSR(n, rp, cols.astype(np.int32), d[rows, cols].copy())


def periodic_5pt(m: int, shift: float = 0.0) -> CSR:
    """Periodic m x m grid, stencil [-1; -1 4+shift -1; -1] (circulant)."""
    n = m * m
    d = np.zeros((n, n))
    for j in range(m):
        for i in range(m):
            r = i + m * j
            d[r, r] += 4.0 + shift
            for (di, dj) in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                c = (i + di) % m + m * ((j + dj) % m)
                d[r, c] += -1.0
    return csr_from_dense(d)


def graph_csr(n: int, edges, weights=None, diag: float = 4.0) -> CSR:
    """Symmetric matrix on a graph: off-diagonal -w on each edge, given diagonal."""
    d = np.zeros((n, n))
    for t, (a, b) in enumerate(edges):
        w = 1.0 if weights is None else weights[t]
        d[a, b] = -w
        d[b, a] = -w
    np.fill_diagonal(d, diag)
    return csr_from_dense(d)


def rows_of(A):
    return np.repeat(np.arange(A.n), np.diff(A.row_ptr))
