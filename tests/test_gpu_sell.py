"""The sliced-ELL copy of the level operators (params.spmv_layout = AMG_LAYOUT_SELL, which
keeps it wherever rows are short, whatever the size) against CSR only (AMG_LAYOUT_CSR) on the
same hierarchy; AMG_LAYOUT_AUTO keeps it only for operators larger than the L2 cache (covered
by the full-size random-coefficient parity test).

A row is summed in the order of the two-lanes-per-row CSR kernel (entries 0, 2, 4, ... and
1, 3, 5, ... added at the end) and the PCG dot partials keep the CSR kernel's blocks and
reduction tree, so the two layouts must give the same bits: V-cycle outputs, PCG and GMRES
iterates, iteration counts and residuals.  Sizes cover a ragged last slice (n not a multiple of
32), rows of different lengths within a slice (boundary rows), FP64 and mixed precision.
"""
import numpy as np
import pytest

from paper_2103_10476_gb300 import problems as P
from tests.gpu_common import gpu_params

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


def _pair(amg, A, **kw):
    arg = amg.csr_arg(A.n, np.ascontiguousarray(A.row_ptr, np.int64), np.ascontiguousarray(A.col, np.int32),
                      np.ascontiguousarray(A.val, np.float64))
    c0 = amg.amg_launch_count()
    ha = amg.amg_setup(arg, None, gpu_params(amg, spmv_layout=amg.AMG_LAYOUT_SELL, **kw))
    c1 = amg.amg_launch_count()
    hc = amg.amg_setup(arg, None, gpu_params(amg, spmv_layout=amg.AMG_LAYOUT_CSR, **kw))
    c2 = amg.amg_launch_count()
    # the copy's layout, scan and fill kernels ran for the first handle only (one level or more)
    if amg.amg_num_levels(ha) > 1:
        assert (c1 - c0) - (c2 - c1) >= 3
    return ha, hc


# Sizes: the fine level must keep two lanes per row (at least two 128-row blocks per SM, else
# the product plan widens its rows and no level gets the copy); 35^3 has ragged slices, 40^3 none.
CASES = [
    ("stretched35", lambda: P.stretched_box(35, 1.1), dict(theta=0.02, variants=3, max_coarse=200)),
    ("stretched40", lambda: P.stretched_box(40, 1.1), dict(theta=0.02, variants=0, max_coarse=200)),
    ("randcoef35", lambda: P.random_coefficient_cube(35, 2, 3.0), dict(theta=0.02, variants=3, max_coarse=200)),
]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_sell_and_csr_give_the_same_bits(amg, name, make, kw, precision):
    A = make()
    assert A.n % 32 != 0 or name == "stretched40"
    ha, hc = _pair(amg, A, precision=precision, **kw)
    assert amg.amg_num_levels(ha) == amg.amg_num_levels(hc) > 1
    # one V-cycle
    r = P.rhs_uniform(A.n, 21)
    za, zc = np.zeros(A.n), np.zeros(A.n)
    amg.amg_vcycle(ha, r, za)
    amg.amg_vcycle(hc, r, zc)
    assert np.array_equal(za, zc)
    # whole PCG solves
    b = P.rhs_uniform(A.n, 22)
    xa, xc = np.zeros(A.n), np.zeros(A.n)
    ia = amg.amg_solve(ha, b, xa, 1e-10)
    ic = amg.amg_solve(hc, b, xc, 1e-10)
    amg.amg_free(ha)
    amg.amg_free(hc)
    assert ia.status == ic.status == 0
    assert ia.iters == ic.iters and ia.relres_true == ic.relres_true
    assert np.array_equal(xa, xc)


def test_sell_gmres_same_bits(amg):
    A = P.convection_diffusion_box(36)
    ha, hc = _pair(amg, A, theta=0.05, variants=3, krylov=1, max_coarse=200)
    b = P.rhs_uniform(A.n, 5)
    xa, xc = np.zeros(A.n), np.zeros(A.n)
    ia = amg.amg_solve(ha, b, xa, 1e-9)
    ic = amg.amg_solve(hc, b, xc, 1e-9)
    amg.amg_free(ha)
    amg.amg_free(hc)
    assert ia.status == ic.status == 0 and ia.iters == ic.iters
    assert np.array_equal(xa, xc)


def test_sell_single_level_and_bad_layout(amg):
    # a hierarchy of one level has no V-cycle products: the layouts coincide trivially
    A = P.stretched_box(6, 1.1)
    ha, hc = _pair(amg, A, theta=0.02, max_coarse=500)
    assert amg.amg_num_levels(ha) == 1
    b = P.rhs_uniform(A.n, 1)
    xa, xc = np.zeros(A.n), np.zeros(A.n)
    assert amg.amg_solve(ha, b, xa, 1e-10).iters == amg.amg_solve(hc, b, xc, 1e-10).iters
    assert np.array_equal(xa, xc)
    amg.amg_free(ha)
    amg.amg_free(hc)
    arg = amg.csr_arg(A.n, np.ascontiguousarray(A.row_ptr, np.int64), np.ascontiguousarray(A.col, np.int32),
                      np.ascontiguousarray(A.val, np.float64))
    h, st = amg.amg_setup_status(arg, None, gpu_params(amg, spmv_layout=7))
    assert h is None and st == amg.AMG_ERR_INVALID_ARG
