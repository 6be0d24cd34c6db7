"""Operators with a few very long rows against the oracle.

Aggregation that stalls leaves coarse levels where a handful of rows couple to every other row
(7,004 entries in a 7,004-row level of the 128^3 random-coefficient cube, mean 4.5).  The
library sums such rows with a block each and the rest with its row tiles; every mode of the
product (plain, residual, Chebyshev step, prolongation, the PCG product with its dot product,
the power method) must keep the oracle's results.

* An arrow-bordered Laplacian: the 27-point Laplacian on 16^3 nodes with its first row and
  column coupled to every node (4,096 entries in row 0): the fine level itself has a long row,
  so the PCG product (with its dot product) and the power method of traditional SA (lambda
  estimated, not fixed) run the long-row path.  Bars: the whole hierarchy (integer
  structures bit-exact, values within VAL_TOL), PCG iterations by the borderline rule,
  solutions within SOL_TOL.
* The 56^3 random-coefficient cube, whose coarse levels 3 and 4 hold rows of 562-835 entries
  (mean 24-38): covered with the same bars in tests/test_gpu_coarse.py.
"""
import numpy as np
import pytest

from paper_2103_10476_gb300 import problems as P
from tests.gpu_common import SOL_TOL, compare_hierarchies, gpu_setup, iterations_agree

pytestmark = pytest.mark.gpu

TOL = 1e-8


@pytest.fixture(scope="module")
def amg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2103_10476_gb300 import build
    build.build()
    from paper_2103_10476_gb300 import amg as m
    return m


def arrow_laplacian(N: int, eps: float):
    """The 27-point Laplacian on N^3 nodes plus -eps on row 0 and column 0 against every other
    node; the diagonal of row 0 is raised by eps (n - 1) + 1, so the matrix stays SPD
    (diagonally dominant in row 0, and each other row gains one entry of magnitude eps, with
    its diagonal raised by eps)."""
    import scipy.sparse as sp
    L = P.laplace_cube(N).to_scipy().tolil()
    n = L.shape[0]
    for j in range(1, n):
        L[0, j] = L[0, j] - eps
        L[j, 0] = L[j, 0] - eps
        L[j, j] = L[j, j] + eps
    L[0, 0] = L[0, 0] + eps * (n - 1) + 1.0
    M = sp.csr_matrix(L)
    M.sort_indices()
    return P.CSR(n, M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64))


@pytest.mark.parametrize("variants,theta", [(0, 0.0), (0, 0.02), (3, 0.02)], ids=["trad-th0", "trad", "1norm+offlmp"])
def test_arrow_matrix_matches_oracle(amg, oracle_lib, variants, theta):
    A = arrow_laplacian(16, 1e-3)
    assert np.diff(A.row_ptr).max() == A.n
    b = P.rhs_uniform(A.n, 11)
    kw = dict(theta=theta, variants=variants, max_coarse=60)
    oh, ost = oracle_lib.setup(A, **kw)
    assert ost == 0
    h, st = gpu_setup(A, **kw)
    assert st == 0, amg.amg_last_error()
    try:
        bad = compare_hierarchies(h, oh)
        assert not bad, bad[:5]
        x = np.zeros(A.n)
        info = amg.amg_solve(h, b, x, TOL)
        xo, oinfo, _ = oh.solve(b, TOL)
        assert info.status == 0
        assert iterations_agree(oracle_lib, A, kw, b, TOL, info.iters, oinfo.iters), (info.iters, oinfo.iters)
        assert np.linalg.norm(x - xo) <= SOL_TOL * np.linalg.norm(xo)
        assert info.relres_true <= TOL
    finally:
        amg.amg_free(h)
