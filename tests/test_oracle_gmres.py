"""Pins of the oracle's path for nonsymmetric operators (a GMRES outer iteration, as §3
uses for the wind pressure system): dense LU with partial pivoting, flexible GMRES, and the
symmetrised strength mask.

Each test checks against something other than the code under test: numpy's dense solver,
the minimal-polynomial property of GMRES (an operator with k distinct eigenvalues is solved in
at most k steps), full GMRES reaching the exact solution within n steps, PCG on a symmetric
problem, and the mask's symmetry.
"""
import numpy as np
import pytest

from paper_2103_10476_gb300 import problems as P
from tests.helpers import csr_from_dense, rows_of


def test_lu_with_pivoting_against_numpy(oracle_lib):
    rng = np.random.default_rng(4)
    for n in (1, 5, 37):
        a = rng.standard_normal((n, n))
        if n > 1:
            a[0, 0] = 0.0                      # the first step must exchange rows
        b = rng.standard_normal(n)
        x, st = oracle_lib.lu_solve(a, b)
        assert st == 0
        assert np.allclose(x, np.linalg.solve(a, b), rtol=1e-10, atol=1e-12)
    x, st = oracle_lib.lu_solve(np.zeros((3, 3)), np.ones(3))
    assert st == oracle_lib.ERR_COARSE_NOT_SPD


def test_gmres_minimal_polynomial_steps(oracle_lib):
    # A = S diag(2, 5, 9 repeated) S^-1: its minimal polynomial has degree 3, so GMRES from
    # x = 0 is exact after 3 Arnoldi steps
    rng = np.random.default_rng(9)
    n = 24
    S = np.eye(n) + 0.3 * rng.standard_normal((n, n))
    lam = np.array([2.0, 5.0, 9.0])[np.arange(n) % 3]
    a = S @ np.diag(lam) @ np.linalg.inv(S)
    A = csr_from_dense(a)
    b = rng.standard_normal(n)
    x, info = oracle_lib.gmres_plain(A, b, 1e-10, restart=30)
    assert info.status == 0 and info.iters <= 4, info.iters
    assert np.allclose(x, np.linalg.solve(a, b), rtol=1e-8, atol=1e-10)


def test_full_gmres_reaches_the_solution(oracle_lib):
    rng = np.random.default_rng(2)
    n = 30
    a = rng.standard_normal((n, n)) + n ** 0.5 * np.eye(n)
    A = csr_from_dense(a)
    b = rng.standard_normal(n)
    x, info = oracle_lib.gmres_plain(A, b, 1e-12, restart=n)
    assert info.status == 0 and info.iters <= n
    assert np.allclose(x, np.linalg.solve(a, b), rtol=1e-9, atol=1e-11)
    # restarted every 5 steps it still converges (the residual never grows within a cycle)
    x5, info5 = oracle_lib.gmres_plain(A, b, 1e-10, restart=5, max_iter=2000)
    assert info5.status == 0 and info5.iters >= info.iters


def test_fgmres_with_amg_matches_pcg_on_a_symmetric_problem(oracle_lib):
    A = P.stretched_box(12, 1.1)
    b = P.rhs_uniform(A.n, 3)
    kw = dict(theta=0.02, variants=3, max_coarse=40)
    hc, _ = oracle_lib.setup(A, **kw)
    hg, _ = oracle_lib.setup(A, krylov=1, **kw)
    xc, ic, _ = hc.solve(b, 1e-10)
    xg, ig, _ = hg.solve(b, 1e-10)
    assert ic.status == 0 and ig.status == 0
    assert np.linalg.norm(xg - xc) / np.linalg.norm(xc) <= 1e-8
    # on a symmetric operator the symmetrised mask is the mask
    for l in range(hc.nlevels - 1):
        assert np.array_equal(hc.get(l, "strong"), hg.get(l, "strong"))
        assert np.array_equal(hc.get(l, "agg"), hg.get(l, "agg"))


def test_symmetrised_mask_on_a_nonsymmetric_operator(oracle_lib):
    A = P.convection_diffusion_box(9)
    h, st = oracle_lib.setup(A, theta=0.05, krylov=1, max_coarse=40)
    assert st == 0
    s = h.get(0, "strong")
    rows = rows_of(A)
    own = oracle_lib.strength(A, 0.05)
    strong = {(int(r), int(c)) for r, c, f in zip(rows, A.col, s) if f}
    assert all((c, r) in strong for r, c in strong)
    # it is the union of the entry's own test and its transpose's
    tested = {(int(r), int(c)) for r, c, f in zip(rows, A.col, own) if f}
    assert strong == tested | {(c, r) for r, c in tested}
    assert len(strong) > len(tested)           # the operator is nonsymmetric enough to matter
