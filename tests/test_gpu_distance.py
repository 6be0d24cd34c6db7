"""Parity of the CUDA path with the oracle for the distance-Laplacian strength of §3.1 on the
paper's two stand-in meshes (randomly perturbed cube, triaxially graded reaction-diffusion
cube), through amg_setup_coords.

Bars: strength masks, aggregates, every pattern and the coarse coordinates bit-exact (the
distances, reciprocals, sums and means are each rounded once, in the oracle's order);
values within VAL_TOL; PCG iterations by the rule of the other parity tests.
"""
import numpy as np
import pytest

from paper_2103_10476_gb300 import problems as P
from tests.gpu_common import SOL_TOL, compare_hierarchies, gpu_params, iterations_agree

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


def _arg(amg, A):
    return amg.csr_arg(A.n, np.ascontiguousarray(A.row_ptr, np.int64), np.ascontiguousarray(A.col, np.int32),
                       np.ascontiguousarray(A.val, np.float64))


def _setup(amg, A, coords, **kw):
    p = gpu_params(amg, strength=amg.AMG_STRENGTH_DISTANCE, **kw)
    h = amg.C.c_void_p()
    X = None if coords is None else np.ascontiguousarray(coords, np.float64)
    arg = _arg(amg, A)
    st = amg.lib.amg_setup_coords(amg.C.byref(arg), None, None if X is None else X.ctypes.data,
                                  0 if X is None else X.shape[1], amg.C.byref(p), amg.C.byref(h))
    return (h if st == 0 else None), st


CASES = [
    ("perturbed10", lambda: P.perturbed_cube(10, seed=5), dict(theta=0.025, max_coarse=40)),
    ("perturbed13", lambda: P.perturbed_cube(13, seed=9), dict(theta=0.025, max_coarse=60)),
    ("graded1-5-10", lambda: P.graded_cube(1, 5, 10, 1e3, ne=12), dict(theta=0.025, max_coarse=60)),
]


@pytest.mark.parametrize("variants", [0, 1, 2, 8, 15])
@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_distance_hierarchy_and_solve_match_oracle(amg, oracle_lib, name, make, kw, variants):
    A = make()
    X = A.meta["coords"]
    h, st = _setup(amg, A, X, variants=variants, **kw)
    oh, ost = oracle_lib.setup(A, coords=X, strength=1, variants=variants, **kw)
    assert st == ost, (st, ost, amg.amg_last_error())
    if st != 0:
        return
    bad = compare_hierarchies(h, oh)
    for l in range(1, oh.nlevels):
        g, o = amg.amg_export(h, l, "coords"), oh.get(l, "coords")
        if not np.array_equal(g, o):
            bad.append((l, "coords", int((g != o).sum())))
    assert not bad, bad[:8]
    b = P.rhs_uniform(A.n, 11)
    x = np.zeros(A.n)
    info = amg.amg_solve(h, b, x, 1e-10)
    xo, oinfo, ostat = oh.solve(b, 1e-10)
    amg.amg_free(h)
    assert info.status == ostat
    assert iterations_agree(oracle_lib, A, dict(coords=X, strength=1, variants=variants, **kw), b, 1e-10,
                            info.iters, oinfo.iters), (info.iters, oinfo.iters)
    if info.iters == oinfo.iters and ostat == 0:
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= SOL_TOL


def test_distance_strength_errors(amg):
    A = P.perturbed_cube(5)
    h, st = _setup(amg, A, None, theta=0.025)
    assert h is None and st == amg.AMG_ERR_INVALID_ARG
    X = A.meta["coords"].copy()
    X[1] = X[0]
    h, st = _setup(amg, A, X, theta=0.025, max_coarse=1)
    assert h is None and st == amg.AMG_ERR_INVALID_ARG and "coordinates" in amg.lib.amg_last_error().decode()


def test_device_coordinates_match_host(amg):
    import torch
    A = P.perturbed_cube(9)
    X = A.meta["coords"]
    h1, st1 = _setup(amg, A, X, theta=0.025, max_coarse=30)
    p = gpu_params(amg, strength=amg.AMG_STRENGTH_DISTANCE, theta=0.025, max_coarse=30)
    rp, ci, v = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (A.row_ptr, A.col, A.val))
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    h2 = amg.amg_setup_coords(amg.csr_arg(A.n, rp, ci, v), None, Xd, p)
    assert st1 == 0
    for what in ("strong", "agg", "P.v"):
        assert np.array_equal(amg.amg_export(h1, 0, what), amg.amg_export(h2, 0, what)), what
    assert np.array_equal(amg.amg_export(h1, 1, "coords"), amg.amg_export(h2, 1, "coords"))
    amg.amg_free(h1)
    amg.amg_free(h2)


def test_distance_criterion_cuts_iterations_on_perturbed_cube(amg):
    # §3.1's motivation: on the 100:1 perturbed cube the matrix criterion coarsens badly
    A = P.perturbed_cube(16)
    b = P.rhs_uniform(A.n, 3)
    hd, st = _setup(amg, A, A.meta["coords"], theta=0.025, max_coarse=100)
    assert st == 0
    hm, st2 = amg.amg_setup_status(_arg(amg, A), None, gpu_params(amg, theta=0.025, max_coarse=100))
    assert st2 == 0
    xd, xm = np.zeros(A.n), np.zeros(A.n)
    kd = amg.amg_solve(hd, b, xd, 1e-10).iters
    km = amg.amg_solve(hm, b, xm, 1e-10).iters
    amg.amg_free(hd)
    amg.amg_free(hm)
    assert kd < km
