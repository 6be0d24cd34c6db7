"""Several right-hand sides of one system at once (amg_solve_multi) against each column solved
alone with amg_solve on the same hierarchy, and against the oracle.

Each column runs the arithmetic of amg_solve: the column's share of every sparse product is
summed by the same lanes in the same order, and every dot product uses the same blocks and
the same fixed-order sums, so iteration counts must agree and solutions to rounding.
"""
import numpy as np
import pytest

from paper_2103_10476_gb300 import problems as P
from tests.gpu_common import SOL_TOL, gpu_params, iterations_agree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2103_10476_gb300 import build
    build.build()
    from paper_2103_10476_gb300 import amg as m
    return m


def _setup(amg, A, **kw):
    arg = amg.csr_arg(A.n, np.ascontiguousarray(A.row_ptr, np.int64), np.ascontiguousarray(A.col, np.int32),
                      np.ascontiguousarray(A.val, np.float64))
    return amg.amg_setup(arg, None, gpu_params(amg, **kw))


@pytest.mark.parametrize("layout", ["auto", "sell"])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("k", [1, 3, 8])
def test_multi_equals_each_column_alone(amg, precision, k, layout):
    # layout "sell": every short-row level carries its sliced-ELL copy, which both the single
    # column's products and the block products then read
    A = P.stretched_box(18, 1.1)
    lay = amg.AMG_LAYOUT_SELL if layout == "sell" else amg.AMG_LAYOUT_AUTO
    h = _setup(amg, A, theta=0.02, variants=3, precision=precision, max_coarse=40, spmv_layout=lay)
    B = np.stack([P.rhs_uniform(A.n, 100 + j) for j in range(k)])
    X = np.zeros_like(B)
    st, infos = amg.amg_solve_multi(h, B, X, 1e-8)
    assert st == 0
    for j in range(k):
        xa = np.zeros(A.n)
        ia = amg.amg_solve(h, B[j], xa, 1e-8)
        assert infos[j].status == 0 and infos[j].relres_true <= 1e-8
        assert infos[j].iters == ia.iters, (j, infos[j].iters, ia.iters)
        assert np.linalg.norm(X[j] - xa) / np.linalg.norm(xa) <= 1e-12, j
    amg.amg_free(h)


@pytest.mark.parametrize("precision", [0, 1])
def test_multi_columns_match_oracle(amg, oracle_lib, precision):
    # every column against the oracle's solve of that right-hand side: FP64 iterations by the
    # borderline rule and solutions within SOL_TOL; mixed within one iteration and 1e-6
    A = P.random_coefficient_cube(14, 6, 2.0)
    kw = dict(theta=0.02, variants=3, max_coarse=40)
    h = _setup(amg, A, precision=precision, **kw)
    k = 5
    B = np.stack([P.rhs_uniform(A.n, 500 + j) for j in range(k)])
    X = np.zeros_like(B)
    st, infos = amg.amg_solve_multi(h, B, X, 1e-8)
    amg.amg_free(h)
    assert st == 0
    oh, ost = oracle_lib.setup(A, **kw)
    assert ost == 0
    for j in range(k):
        xo, oinfo, _ = oh.solve(B[j], 1e-8)
        if precision:
            assert abs(infos[j].iters - oinfo.iters) <= 1, (j, infos[j].iters, oinfo.iters)
            assert np.linalg.norm(X[j] - xo) / np.linalg.norm(xo) <= 1e-6
        else:
            assert iterations_agree(oracle_lib, A, kw, B[j], 1e-8, infos[j].iters, oinfo.iters), j
            assert np.linalg.norm(X[j] - xo) / np.linalg.norm(xo) <= SOL_TOL


def test_multi_zero_column_limit_and_device_arrays(amg):
    import torch
    A = P.random_coefficient_cube(12, 3, 2.0)
    h = _setup(amg, A, theta=0.02, variants=3, max_coarse=60)
    B = np.stack([P.rhs_uniform(A.n, 7), np.zeros(A.n), P.rhs_uniform(A.n, 8)])
    X = np.full_like(B, 5.0)
    st, infos = amg.amg_solve_multi(h, B, X, 1e-8)
    assert st == 0 and infos[1].iters == 0 and not X[1].any()
    Bd = torch.from_numpy(B).cuda()
    Xd = torch.zeros_like(Bd)
    st2, infos2 = amg.amg_solve_multi(h, Bd, Xd, 1e-8)
    assert st2 == 0 and np.array_equal(Xd.cpu().numpy(), X)
    assert [i.iters for i in infos2] == [i.iters for i in infos]
    amg.amg_free(h)
    # an iteration limit stops every running column with NOT_CONVERGED and its last iterate
    h = _setup(amg, A, theta=0.02, variants=3, max_coarse=60, max_iter=2)
    X = np.zeros_like(B)
    st, infos = amg.amg_solve_multi(h, B, X, 1e-8)
    assert st == amg.AMG_ERR_NOT_CONVERGED
    assert infos[0].iters == 2 and infos[0].status == amg.AMG_ERR_NOT_CONVERGED and infos[1].status == 0
    xa = np.zeros(A.n)
    ia = amg.amg_solve(h, B[2], xa, 1e-8)
    assert ia.iters == 2 and np.linalg.norm(X[2] - xa) / np.linalg.norm(xa) <= 1e-12
    amg.amg_free(h)
