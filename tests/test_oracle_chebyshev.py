"""Pins of the oracle's Chebyshev smoother (§3.1: degree 2 in D^-1 A on [lambda*/10, lambda*])
and of the V-cycle that applies it (Algorithm 1), against closed forms built with numpy.

From any start x0, m steps of Chebyshev acceleration for A x = f with M = D^-1 A leave the
error e_m = p_m(M) e_0, where p_m is the residual polynomial of the interval [a, b]:

    p_m(t) = T_m((b + a - 2t)/(b - a)) / T_m((b + a)/(b - a)),     T_m the Chebyshev polynomial.

The reference side evaluates p_m on the eigenvalues of the symmetric D^-1/2 A D^-1/2 (numpy's
eigh) and T_m with numpy's Chebyshev series; it never runs the three-term recurrence.  A wrong
recurrence coefficient, an interval end, an off-by-one degree or the boost factor applied twice
moves the result far outside the tolerance.
"""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

from paper_2103_10476_gb300 import problems as P
from tests.helpers import csr_from_dense


def _spd(n, seed, cond=1e3):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    ev = np.geomspace(1.0, cond, n)
    a = (Q * ev) @ Q.T
    s = np.exp(rng.uniform(-1.0, 1.0, n))        # a diagonal far from constant: D != c I
    return s[:, None] * a * s[None, :]


def _closed_form(a, f, x0, lam, degree, ratio, boost):
    """x after `degree` Chebyshev steps, from the residual polynomial on the spectrum of D^-1 A."""
    d = np.diag(a)
    dh = 1.0 / np.sqrt(d)
    S = dh[:, None] * a * dh[None, :]
    mu, V = np.linalg.eigh(S)
    hi = boost * lam
    lo = hi / ratio
    Tm = np.zeros(degree + 1)
    Tm[-1] = 1.0
    p = npcheb.chebval((hi + lo - 2.0 * mu) / (hi - lo), Tm) / npcheb.chebval((hi + lo) / (hi - lo), Tm)
    xs = np.linalg.solve(a, f)
    # e_m = D^-1/2 p(S) D^1/2 e_0
    e0 = xs - x0
    em = dh * (V @ (p * (V.T @ (e0 / dh))))
    return xs - em


def _lam_max(a):
    d = np.diag(a)
    dh = 1.0 / np.sqrt(d)
    return float(np.linalg.eigvalsh(dh[:, None] * a * dh[None, :])[-1])


@pytest.mark.parametrize("degree", [1, 2, 3])
@pytest.mark.parametrize("boost", [1.0, 1.1])
@pytest.mark.parametrize("ratio", [10.0, 30.0])
def test_chebyshev_equals_residual_polynomial(oracle_lib, degree, boost, ratio):
    n = 24
    a = _spd(n, 7 + degree)
    A = csr_from_dense(a)
    rng = np.random.default_rng(degree)
    f = rng.uniform(-1, 1, n)
    lmax = _lam_max(a)
    for lam in (lmax, 0.8 * lmax):                       # the exact top, and an underestimate
        for x0 in (np.zeros(n), rng.normal(size=n)):
            x, st = oracle_lib.chebyshev_apply(A, lam, degree, x0=x0, f=f, ratio=ratio, boost=boost)
            assert st == 0
            ref = _closed_form(a, f, x0, lam, degree, ratio, boost)
            assert np.linalg.norm(x - ref) <= 1e-11 * np.linalg.norm(ref), (lam, degree, boost, ratio)


def test_chebyshev_degree_and_interval_are_distinguishable(oracle_lib):
    # the pin would catch the plausible slips: degree m - 1 or m + 1, [lambda/10, lambda] vs the
    # boosted interval, a transposed interval
    n = 24
    a = _spd(n, 3)
    A = csr_from_dense(a)
    f = np.random.default_rng(0).uniform(-1, 1, n)
    lam = _lam_max(a)
    x, _ = oracle_lib.chebyshev_apply(A, lam, 2, f=f, ratio=10.0, boost=1.1)
    ref = _closed_form(a, f, np.zeros(n), lam, 2, 10.0, 1.1)
    for wrong in (_closed_form(a, f, np.zeros(n), lam, 1, 10.0, 1.1),
                  _closed_form(a, f, np.zeros(n), lam, 3, 10.0, 1.1),
                  _closed_form(a, f, np.zeros(n), lam, 2, 10.0, 1.0),
                  _closed_form(a, f, np.zeros(n), lam, 2, 10.0, 1.21)):
        assert np.linalg.norm(wrong - ref) > 1e-6 * np.linalg.norm(ref)
    assert np.linalg.norm(x - ref) <= 1e-11 * np.linalg.norm(ref)


def test_chebyshev_reduces_energy_error_inside_interval(oracle_lib):
    # with the interval covering the whole spectrum of D^-1 A (boost >= 1 on the exact top), the
    # polynomial is at most 1/T_m((b+a)/(b-a)) < 1 in magnitude on [a, b] and at most 1 below a,
    # so the A-norm error never grows
    n = 30
    a = _spd(n, 11, cond=1e4)
    A = csr_from_dense(a)
    rng = np.random.default_rng(5)
    f = rng.uniform(-1, 1, n)
    xs = np.linalg.solve(a, f)
    x0 = rng.normal(size=n)
    x, _ = oracle_lib.chebyshev_apply(A, _lam_max(a), 2, x0=x0, f=f, ratio=10.0, boost=1.0)
    e0, e2 = xs - x0, xs - x
    assert e2 @ a @ e2 <= e0 @ a @ e0


@pytest.mark.parametrize("boost", [1.0, 1.1])
def test_two_level_vcycle_is_algorithm1_with_the_chebyshev_smoother(oracle_lib, boost):
    # Algorithm 1 on two levels from u = 0: pre-smooth, restrict the residual, solve the
    # coarsest level exactly, prolongate and add, post-smooth.  Every step is formed with
    # numpy from the exported level (A, P, R, lambda*) and the closed-form smoother.
    A = P.random_coefficient_cube(7, 4)
    h, st = oracle_lib.setup(A, theta=0.02, variants=3, max_coarse=40, max_levels=2, cheb_boost=boost)
    assert st == 0 and h.nlevels == 2
    L0 = h.level(0)
    L1 = h.level(1)
    a = L0["A"].to_dense()
    Pm = L0["P"].to_dense(L0["nagg"])
    Rm = L0["R"].to_dense(A.n)
    ac = L1["A"].to_dense()
    lam = L0["lambda_cheb"]
    f = P.rhs_uniform(A.n, 3)
    u = _closed_form(a, f, np.zeros(A.n), lam, 2, 10.0, boost)
    uc = np.linalg.solve(ac, Rm @ (f - a @ u))
    u = u + Pm @ uc
    u = _closed_form(a, f, u, lam, 2, 10.0, boost)
    got = h.vcycle(f)
    assert np.linalg.norm(got - u) <= 1e-10 * np.linalg.norm(u)
