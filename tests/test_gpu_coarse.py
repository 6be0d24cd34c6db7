"""The coarsest-level solve (§3.1: a direct solve on the coarsest level) on the GPU against the
oracle's dense Cholesky, for the three ways the library solves the coarsest level.

* Aggregation that stalls: on random-coefficient cubes at theta = 0.02 nothing is strong any
  more below some level, almost every vertex stays a singleton and the hierarchy ends on a
  large, sparse operator whose Jacobi-scaled form is close to the identity (822 rows, scaled
  condition number 1.11, on the 56^3 cube).  By default (AMG_COARSE_AUTO) the V-cycle solves it
  with a fixed Chebyshev polynomial in D^-1 A; with AMG_COARSE_INVERSE it applies an inverse
  formed by conjugate gradients on all columns of the Jacobi-scaled operator.  Bars for both:
  the whole hierarchy as in the other parity tests, the V-cycle within 1e-12 of the oracle's,
  PCG iterations by the borderline rule, solutions within SOL_TOL; for the polynomial, its
  interval must hold the whole spectrum of D^-1 A (numpy's eigvalsh of the oracle's operator).
* A single-level hierarchy of more than 512 rows (its V-cycle is the coarse solve alone): a
  shifted Laplacian (scaled spectrum narrow: the polynomial), the plain Laplacian (scaled
  condition number ~100: a polynomial would need hundreds of steps, so the CG inverse), and a
  dense operator (the dense path); PCG must stop after one iteration with the solution of
  scipy's direct solver.
* The batch engine applies inverses: a handle set up with the polynomial joins a batch, which
  forms its inverse; the batch solve must agree with amg_solve's.  amg_solve_multi runs the
  polynomial on its block of columns.
"""
import numpy as np
import pytest

from paper_2103_10476_gb300 import problems as P
from tests.gpu_common import SOL_TOL, compare_hierarchies, gpu_setup, iterations_agree

pytestmark = pytest.mark.gpu

TOL = 1e-8
KW = dict(theta=0.02, variants=["1norm", "offlmp"])


@pytest.fixture(scope="module")
def amg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2103_10476_gb300 import build
    build.build()
    from paper_2103_10476_gb300 import amg as m
    return m


@pytest.fixture(scope="module")
def stalled(oracle_lib):
    A = P.random_coefficient_cube(56, 2, 3.0)
    b = P.rhs_uniform(A.n, 2)
    oh, st = oracle_lib.setup(A, **KW)
    assert st == 0
    return A, b, oh


def test_stalled_aggregation_ends_on_a_large_well_conditioned_level(stalled):
    A, b, oh = stalled
    L = oh.nlevels - 1
    n = len(oh.get(L, "A.rp")) - 1
    assert n > 512
    lv = oh.level(L)
    d = lv["A"].to_dense()
    assert np.count_nonzero(d) * 8 <= n * n              # sparse: the CG path applies
    s = 1.0 / np.sqrt(np.diag(d))
    ev = np.linalg.eigvalsh(s[:, None] * d * s[None, :])
    assert ev[0] > 0.0 and ev[-1] / ev[0] < 2.0           # Jacobi-scaled: close to the identity


def _scaled_spectrum(oh):
    d = oh.level(oh.nlevels - 1)["A"].to_dense()
    s = 1.0 / np.sqrt(np.diag(d))
    return np.linalg.eigvalsh(s[:, None] * d * s[None, :])


@pytest.mark.parametrize("coarse", ["auto", "inverse"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_stalled_hierarchy_matches_oracle(amg, oracle_lib, stalled, precision, coarse):
    A, b, oh = stalled
    prec = amg.AMG_FP64 if precision == "fp64" else amg.AMG_MIXED
    cs = amg.AMG_COARSE_AUTO if coarse == "auto" else amg.AMG_COARSE_INVERSE
    h, st = gpu_setup(A, precision=prec, coarse_solve=cs, **KW)
    assert st == 0, amg.amg_last_error()
    try:
        deg, theta, delta, check = amg.amg_coarse_solver(h)
        if coarse == "auto":
            ev = _scaled_spectrum(oh)
            assert 2 <= deg <= 40 and 0.0 <= check <= 1e-12, (deg, check)
            assert theta - delta < ev[0] and ev[-1] < theta + delta, (theta - delta, theta + delta, ev[0], ev[-1])
        else:
            assert deg == 0
        if precision == "fp64":
            bad = compare_hierarchies(h, oh)
            assert not bad, bad[:5]
            # one V-cycle: the coarse solve through the inverse formed by CG
            z = np.zeros(A.n)
            amg.amg_vcycle(h, b, z)
            zo = oh.vcycle(b)
            assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)
        x = np.zeros(A.n)
        info = amg.amg_solve(h, b, x, TOL)
        xo, oinfo, ost = oh.solve(b, TOL)
        assert info.status == 0 and ost == 0
        if precision == "fp64":
            assert iterations_agree(oracle_lib, A, KW, b, TOL, info.iters, oinfo.iters), (info.iters, oinfo.iters)
            assert np.linalg.norm(x - xo) <= SOL_TOL * np.linalg.norm(xo)
        else:
            assert abs(info.iters - oinfo.iters) <= 1
            assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)
        assert info.relres_true <= TOL
    finally:
        amg.amg_free(h)


def _one_level(amg, A):
    b = P.rhs_uniform(A.n, 7)
    h, st = gpu_setup(A, theta=0.0, max_levels=1)
    assert st == 0, amg.amg_last_error()
    try:
        assert amg.amg_num_levels(h) == 1
        x = np.zeros(A.n)
        info = amg.amg_solve(h, b, x, 1e-10)
        deg = amg.amg_coarse_solver(h)[0]
    finally:
        amg.amg_free(h)
    import scipy.sparse.linalg as spla
    xs = spla.spsolve(A.to_scipy().tocsc(), b)
    return info, x, xs, deg


def test_single_level_diagonally_dominant_takes_one_iteration(amg):
    # 27-point Laplacian on 10^3 nodes plus a diagonal shift of 20 times its largest entry
    A = P.laplace_cube(10)
    shift = 20.0 * np.abs(A.val).max()
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    A.val[rows == A.col] += shift
    info, x, xs, deg = _one_level(amg, A)
    assert deg > 0                                   # narrow scaled spectrum: the polynomial
    assert info.status == 0 and info.iters == 1
    assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)


def test_single_level_laplacian(amg):
    # the plain 27-point Laplacian on 10^3 nodes (scaled condition number ~100)
    A = P.laplace_cube(10)
    info, x, xs, deg = _one_level(amg, A)
    assert deg == 0                                  # too wide for a short polynomial
    assert info.status == 0 and info.iters == 1
    assert np.linalg.norm(x - xs) <= 1e-11 * np.linalg.norm(xs)


def test_single_level_dense_operator_takes_the_dense_path(amg):
    # a dense SPD operator of 600 rows (more than one entry in eight stored): the dense path
    from tests.helpers import csr_from_dense
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.normal(size=(600, 600)))
    a = (Q * np.geomspace(1.0, 1e3, 600)) @ Q.T
    A = csr_from_dense(a)
    info, x, xs, deg = _one_level(amg, A)
    assert deg == 0
    assert info.status == 0 and info.iters == 1
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)


def test_batch_forms_the_inverse_of_a_polynomial_handle(amg, stalled):
    # the handle solves its coarsest level with the polynomial; joining a batch forms the
    # inverse the engine applies.  Both are the exact coarse solve to ~1e-16, so the batch solve
    # (FP64 here) agrees with amg_solve to a rounding-level difference in the preconditioner.
    A, b, _ = stalled
    h, st = gpu_setup(A, **KW)
    assert st == 0, amg.amg_last_error()
    try:
        assert amg.amg_coarse_solver(h)[0] > 0
        x = np.zeros(A.n)
        info = amg.amg_solve(h, b, x, TOL)
        bt = amg.amg_batch_create([h])
        try:
            xb = np.zeros(A.n)
            stb, infos = amg.amg_batch_solve(bt, [b], [xb], TOL)
            assert stb == 0 and infos[0].status == 0
            assert abs(infos[0].iters - info.iters) <= 1, (infos[0].iters, info.iters)
            assert infos[0].relres_true <= TOL and info.relres_true <= TOL
            if infos[0].iters == info.iters:
                assert np.linalg.norm(xb - x) <= 1e-9 * np.linalg.norm(x)
        finally:
            amg.amg_batch_free(bt)
    finally:
        amg.amg_free(h)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_multi_runs_the_polynomial_on_every_column(amg, stalled, precision):
    A, b, _ = stalled
    prec = amg.AMG_FP64 if precision == "fp64" else amg.AMG_MIXED
    h, st = gpu_setup(A, precision=prec, **KW)
    assert st == 0, amg.amg_last_error()
    try:
        assert amg.amg_coarse_solver(h)[0] > 0
        B = np.stack([P.rhs_uniform(A.n, 30 + j) for j in range(3)])
        X = np.zeros_like(B)
        stm, infos = amg.amg_solve_multi(h, B, X, TOL)
        assert stm == 0
        for j in range(3):
            xa = np.zeros(A.n)
            ia = amg.amg_solve(h, B[j], xa, TOL)
            assert infos[j].status == 0 and infos[j].relres_true <= TOL
            assert abs(infos[j].iters - ia.iters) <= 1, (j, infos[j].iters, ia.iters)
            if infos[j].iters == ia.iters:
                bar = 1e-9 if precision == "fp64" else 1e-5
                assert np.linalg.norm(X[j] - xa) <= bar * np.linalg.norm(xa), j
    finally:
        amg.amg_free(h)
