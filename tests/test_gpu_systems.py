"""Parity of the CUDA path with the oracle for systems of PDEs (block_size unknowns per node,
nullspace_dim near-null-space vectors): 3D elasticity with its six rigid-body modes, the
component constants, and two interleaved copies of a scalar operator.

Bars: node aggregates, roots, strength and removal masks and every pattern bit-exact; values
(QR tentative prolongator, filtered matrix, P, R, coarse operators and near-null spaces) within
VAL_TOL; PCG iterations by the borderline rule; solutions within SOL_TOL; the same statuses for
unsupported cases.
"""
import numpy as np
import pytest

from paper_2103_10476_gb300 import problems as P
from tests.gpu_common import SOL_TOL, compare_hierarchies, gpu_params

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


def _setup(amg, A, B, **kw):
    ns = None if B is None else np.ascontiguousarray(B, np.float64).reshape(-1)
    return amg.amg_setup_status(_arg(amg, A), ns, gpu_params(amg, **kw))


def _box(nx, ny, nz):
    return P.elasticity_box(np.ones(nx), np.ones(ny), np.ones(nz))


def _iters_agree(oracle_lib, A, B, kw, b, tol, kg, ko):
    # identical, or within 2 when the oracle's own true residual at the smaller count is
    # already within twice the tolerance (a borderline stop)
    if kg == ko:
        return True
    if abs(kg - ko) > 2:
        return False
    hk, _ = oracle_lib.setup(A, nullspace=B, max_iter=min(kg, ko), **kw)
    _, info, _ = hk.solve(b, tol)
    return info.relres_true <= 2.0 * tol


CASES = [
    ("elast6-rbm-t0.02", lambda: _box(6, 6, 6), "rbm", dict(theta=0.02, max_coarse=60)),
    ("elast8x6x5-rbm-t0", lambda: _box(8, 6, 5), "rbm", dict(theta=0.0, max_coarse=60)),
    ("elast10-rbm-t0.05", lambda: _box(10, 10, 10), "rbm", dict(theta=0.05, max_coarse=100)),
    ("elast9-const-t0.02", lambda: _box(9, 8, 7), "const", dict(theta=0.02, max_coarse=60)),
]


@pytest.mark.parametrize("name,make,ns,kw", CASES, ids=[c[0] for c in CASES])
def test_systems_hierarchy_and_solve_match_oracle(amg, oracle_lib, name, make, ns, kw):
    A = make()
    B = A.meta["rbm"] if ns == "rbm" else None
    k = 6 if ns == "rbm" else 3
    kw = dict(kw, block_size=3, nullspace_dim=k)
    h, st = _setup(amg, A, B, **kw)
    oh, ost = oracle_lib.setup(A, nullspace=B, **kw)
    assert st == ost == 0, (st, ost, amg.amg_last_error())
    bad = compare_hierarchies(h, oh)
    assert not bad, bad[:8]
    b = P.rhs_uniform(A.n, 4)
    x = np.zeros(A.n)
    info = amg.amg_solve(h, b, x, 1e-10)
    amg.amg_free(h)
    xo, oinfo, ostat = oh.solve(b, 1e-10)
    assert info.status == ostat == 0
    assert _iters_agree(oracle_lib, A, B, kw, b, 1e-10, info.iters, oinfo.iters), (info.iters, oinfo.iters)
    if info.iters == oinfo.iters:
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= SOL_TOL
    assert np.linalg.norm(b - A.to_scipy() @ x) / np.linalg.norm(b) <= 1.01e-10


def test_systems_mixed_precision(amg, oracle_lib):
    A = _box(10, 8, 8)
    B = A.meta["rbm"]
    kw = dict(theta=0.02, max_coarse=80, block_size=3, nullspace_dim=6)
    h, st = _setup(amg, A, B, precision=amg.AMG_MIXED, **kw)
    assert st == 0
    b = P.rhs_uniform(A.n, 5)
    x = np.zeros(A.n)
    info = amg.amg_solve(h, b, x, 1e-8)
    amg.amg_free(h)
    oh, _ = oracle_lib.setup(A, nullspace=B, **kw)
    xo, oinfo, _ = oh.solve(b, 1e-8)
    assert info.status == 0 and abs(info.iters - oinfo.iters) <= 1, (info.iters, oinfo.iters)
    assert np.linalg.norm(b - A.to_scipy() @ x) / np.linalg.norm(b) <= 1.01e-8
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-6


def _interleave(A, copies):
    rows, cols, vals = [], [], []
    r = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    for c in range(copies):
        rows.append(copies * r + c)
        cols.append(copies * A.col.astype(np.int64) + c)
        vals.append(A.val)
    rows, cols, vals = (np.concatenate(x) for x in (rows, cols, vals))
    o = np.lexsort((cols, rows))
    n = copies * A.n
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, rows[o] + 1, 1)
    return P.CSR(n, np.cumsum(rp), cols[o].astype(np.int32), vals[o])


def test_decoupled_system_matches_oracle(amg, oracle_lib):
    A2 = _interleave(P.stretched_box(10, 1.1), 2)
    kw = dict(theta=0.02, block_size=2, nullspace_dim=2, max_coarse=80)
    h, st = _setup(amg, A2, None, **kw)
    oh, ost = oracle_lib.setup(A2, **kw)
    assert st == ost == 0
    bad = compare_hierarchies(h, oh)
    amg.amg_free(h)
    assert not bad, bad[:8]


def test_systems_unsupported_and_invalid(amg, oracle_lib):
    A = _box(4, 4, 4)
    B = A.meta["rbm"]
    for kw, want in ((dict(variants=1), amg.AMG_ERR_UNSUPPORTED),
                     (dict(nullspace_dim=9), amg.AMG_ERR_INVALID_ARG),
                     (dict(block_size=17), amg.AMG_ERR_INVALID_ARG)):
        args = dict(dict(theta=0.02, block_size=3, nullspace_dim=6), **kw)
        h, st = _setup(amg, A, np.tile(B, (2, 1))[:args["nullspace_dim"]] if args["nullspace_dim"] <= 12 else B,
                       **args)
        assert h is None and st == want, (kw, st)
    # no vectors given and k != bs
    h, st = _setup(amg, A, None, block_size=3, nullspace_dim=6)
    assert h is None and st == amg.AMG_ERR_INVALID_ARG
    # n not a multiple of bs
    S = P.stretched_box(5, 1.1)
    h, st = _setup(amg, S, None, block_size=2, nullspace_dim=2)
    assert h is None and st == amg.AMG_ERR_INVALID_ARG
    # a near-null space whose vectors are dependent on every aggregate (two equal columns):
    # both sides refuse it
    Bd = B.copy()
    Bd[5] = Bd[4]
    kw = dict(theta=0.02, block_size=3, nullspace_dim=6, max_coarse=10)
    h, st = _setup(amg, A, Bd, **kw)
    oh, ost = oracle_lib.setup(A, nullspace=Bd, **kw)
    assert h is None and st == ost == amg.AMG_ERR_UNSUPPORTED


def test_systems_device_nullspace_and_repeat(amg):
    import torch
    A = _box(6, 6, 6)
    B = np.ascontiguousarray(A.meta["rbm"])
    kw = dict(theta=0.02, block_size=3, nullspace_dim=6, max_coarse=60)
    h1, st = _setup(amg, A, B, **kw)
    rp, ci, v = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (A.row_ptr, A.col, A.val))
    Bd = torch.from_numpy(B.reshape(-1)).cuda()
    h2 = amg.amg_setup(amg.csr_arg(A.n, rp, ci, v), Bd, gpu_params(amg, **kw))
    assert st == 0
    for l in range(amg.amg_num_levels(h1)):
        for what in ("A.v", "B"):
            assert np.array_equal(amg.amg_export(h1, l, what), amg.amg_export(h2, l, what)), (l, what)
    b = P.rhs_uniform(A.n, 9)
    x1, x2 = np.zeros(A.n), np.zeros(A.n)
    i1 = amg.amg_solve(h1, b, x1, 1e-10)
    i2 = amg.amg_solve(h2, b, x2, 1e-10)
    amg.amg_free(h1)
    amg.amg_free(h2)
    assert i1.status == i2.status == 0 and i1.iters == i2.iters and np.array_equal(x1, x2)
