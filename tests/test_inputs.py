"""The seeded input generators shared by the tests and the benchmark (no GPU)."""
import numpy as np
import pytest

from paper_2103_10476_gb300 import problems as P


@pytest.mark.parametrize("N", [1, 2, 7, 18])
def test_c_assembly_is_bit_identical_to_numpy(N):
    pairs = [(lambda e: P.stretched_box(N, 1.17, engine=e)),
             (lambda e: P.random_coefficient_cube(N, 11, 2.0, engine=e)),
             (lambda e: P.laplace_cube(N) if e == "numpy" else P.q1_matrix(*([np.full(N + 1, 1.0 / (N + 1))] * 3),
                                                                            engine="c"))]
    for make in pairs:
        a, b = make("numpy"), make("c")
        assert a.n == b.n
        assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
        assert np.array_equal(a.val.view(np.uint64), b.val.view(np.uint64))


def test_c_assembly_neumann_and_anisotropic():
    hx, hy, hz = np.full(3, 0.5), np.array([0.25, 1.0, 2.0, 0.1]), np.linspace(1, 3, 5)
    a = P.q1_matrix(hx, hy, hz, dirichlet=False)
    b = P.q1_matrix(hx, hy, hz, dirichlet=False, engine="c")
    assert np.array_equal(a.col, b.col) and np.array_equal(a.val.view(np.uint64), b.val.view(np.uint64))
    # a pure-Neumann operator annihilates constants (row sums vanish to rounding)
    assert np.abs(b.to_scipy() @ np.ones(b.n)).max() < 1e-12 * np.abs(b.val).max()


def test_serving_stream_shape():
    reqs, ops = P.serving_stream(20.0, rate=200.0)
    t = np.array([r[0] for r in reqs])
    assert abs(len(reqs) / 20.0 - 200.0) < 15.0            # Poisson rate
    assert np.all(np.diff(t) > 0) and t[-1] < 20.0
    repeats = len(reqs) - len(ops)
    assert abs(repeats / len(reqs) - 0.3) < 0.04           # 30% repeat an earlier operator
    Ns = np.array([o[1] for o in ops])
    assert Ns.min() >= 16 and Ns.max() <= 96
    assert abs(np.median(np.log(Ns)) - 0.5 * (np.log(16) + np.log(96))) < 0.1   # log-uniform
    nrhs = np.array([r[2] for r in reqs])
    assert nrhs.min() == 1 and nrhs.max() == 8
    fam = [o[0] for o in ops]
    assert 0.4 < fam.count("stretched") / len(fam) < 0.6
    assert P.serving_stream(20.0)[0] == reqs                # seeded
