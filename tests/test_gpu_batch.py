"""Many systems in one batch (amg_setup_batch / amg_batch_solve) against each system solved
alone (amg_solve on the same hierarchy) and against the oracle.

Every system of a batch runs its own PCG (own scalars, own stopping test) through shared
launches, so a batched result must be the result of that system alone: the same iteration
count (FP64: exactly, or within two when the stop is borderline by the oracle's own residual,
the rule of the single-system parity tests, since the summation order of the dot products
differs; mixed precision: within one) and a solution within SOL_TOL.  With lanes per row chosen from the
mean row length (no timing), a system's rows are computed by the same lanes in the same order
wherever the system sits, so reordering the systems of a batch changes nothing, bit for bit.
"""
import numpy as np
import pytest

from paper_2103_10476_gb300 import problems as P
from tests.gpu_common import SOL_TOL, gpu_params, iterations_agree

pytestmark = pytest.mark.gpu

KW = dict(theta=0.02, variants=3, max_coarse=60)


@pytest.fixture(scope="module")
def amg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2103_10476_gb300 import build
    build.build()
    from paper_2103_10476_gb300 import amg as m
    return m


def _systems():
    # uneven sizes and depths: stretched boxes and random-coefficient cubes, one system small
    # enough to be its own coarsest level (n <= max_coarse), one with a ragged edge
    out = [(P.stretched_box(12, 1.1), 1), (P.random_coefficient_cube(9, 7, 2.0), 2), (P.laplace_cube(3), 3),
           (P.stretched_box(17, 1.15), 4), (P.random_coefficient_cube(14, 8, 2.0), 5), (P.laplace_cube(6), 6),
           (P.stretched_box(8, 1.05), 7), (P.random_coefficient_cube(11, 9, 2.0), 8)]
    return [(A, P.rhs_uniform(A.n, s)) for A, s in out]


def _args(amg, systems):
    keep, As = [], []
    for A, _ in systems:
        rp = np.ascontiguousarray(A.row_ptr, np.int64)
        ci = np.ascontiguousarray(A.col, np.int32)
        v = np.ascontiguousarray(A.val, np.float64)
        keep.append((rp, ci, v))
        As.append(amg.csr_arg(A.n, rp, ci, v))
    return keep, As


def _setup(amg, systems, **kw):
    keep, As = _args(amg, systems)
    return amg.amg_setup_batch(As, None, gpu_params(amg, **kw))


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_each_system_alone(amg, oracle_lib, precision):
    systems = _systems()
    hs = _setup(amg, systems, precision=precision, **KW)
    alone = []
    for h, (A, b) in zip(hs, systems):
        x = np.zeros(A.n)
        alone.append((amg.amg_solve(h, b, x, 1e-8), x))
    bt = amg.amg_batch_create(hs)
    xs = [np.zeros(A.n) for A, _ in systems]
    st, infos = amg.amg_batch_solve(bt, [b for _, b in systems], xs, 1e-8)
    count, levels, rows, gk = amg.amg_batch_info(bt)
    amg.amg_batch_free(bt)
    for h in hs:
        amg.amg_free(h)
    assert st == 0
    assert count == len(systems) and rows == sum(A.n for A, _ in systems) and gk > 0
    for k, ((A, b), (ia, xa), ib, xb) in enumerate(zip(systems, alone, infos, xs)):
        assert ib.status == 0 and ib.relres_true <= 1e-8, (k, ib.status, ib.relres_true)
        assert ib.levels == ia.levels
        if precision:
            assert abs(ib.iters - ia.iters) <= 1, (k, ib.iters, ia.iters)
        else:
            assert iterations_agree(oracle_lib, A, KW, b, 1e-8, ib.iters, ia.iters), (k, ib.iters, ia.iters)
        assert np.linalg.norm(xb - xa) / np.linalg.norm(xa) <= (1e-6 if precision else SOL_TOL), k


def test_batch_iterations_match_oracle(amg, oracle_lib):
    systems = _systems()[:5]
    hs = _setup(amg, systems, **KW)
    xs = [np.zeros(A.n) for A, _ in systems]
    st, infos = amg.amg_solve_batch(hs, [b for _, b in systems], xs, 1e-8)
    for h in hs:
        amg.amg_free(h)
    assert st == 0
    for (A, b), info, x in zip(systems, infos, xs):
        oh, ost = oracle_lib.setup(A, **KW)
        assert ost == 0
        xo, oinfo, _ = oh.solve(b, 1e-8)
        assert iterations_agree(oracle_lib, A, KW, b, 1e-8, info.iters, oinfo.iters), (info.iters, oinfo.iters)
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= SOL_TOL


def test_batch_order_does_not_change_results(amg):
    systems = _systems()
    hs = _setup(amg, systems, precision=1, **KW)
    bs = [b for _, b in systems]
    x1 = [np.zeros(A.n) for A, _ in systems]
    st1, i1 = amg.amg_solve_batch(hs, bs, x1, 1e-8)
    perm = [5, 2, 7, 0, 3, 6, 1, 4]
    x2 = [np.zeros(systems[k][0].n) for k in perm]
    st2, i2 = amg.amg_solve_batch([hs[k] for k in perm], [bs[k] for k in perm], x2, 1e-8)
    for h in hs:
        amg.amg_free(h)
    assert st1 == 0 and st2 == 0
    for j, k in enumerate(perm):
        assert i2[j].iters == i1[k].iters
        assert np.array_equal(x2[j], x1[k]), k


def test_batch_zero_rhs_and_iteration_limit(amg):
    systems = _systems()[:4]
    hs = _setup(amg, systems, max_iter=3, **KW)
    bs = [b.copy() for _, b in systems]
    bs[1][:] = 0.0
    xs = [np.full(A.n, 7.0) for A, _ in systems]
    st, infos = amg.amg_solve_batch(hs, bs, xs, 1e-8)
    for h in hs:
        amg.amg_free(h)
    assert st == amg.AMG_ERR_NOT_CONVERGED
    assert infos[1].status == 0 and infos[1].iters == 0 and not xs[1].any()
    for k in (0, 2, 3):
        if systems[k][0].n > 60:
            assert infos[k].status == amg.AMG_ERR_NOT_CONVERGED and infos[k].iters == 3


def test_batch_device_vectors(amg):
    import torch
    systems = _systems()[:3]
    hs = _setup(amg, systems, **KW)
    bs = [torch.from_numpy(b).cuda() for _, b in systems]
    xs = [torch.zeros(A.n, dtype=torch.float64, device="cuda") for A, _ in systems]
    xh = [np.zeros(A.n) for A, _ in systems]
    st, infos = amg.amg_solve_batch(hs, bs, xs, 1e-8)
    st2, _ = amg.amg_solve_batch(hs, [b for _, b in systems], xh, 1e-8)
    for h in hs:
        amg.amg_free(h)
    assert st == 0 and st2 == 0
    for a, b in zip(xs, xh):
        assert np.array_equal(a.cpu().numpy(), b)


def test_setup_batch_reports_failing_system(amg):
    systems = _systems()[:3]
    A = P.laplace_cube(5)
    bad = P.CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val.copy())
    # an asymmetric structure error: the first row loses its diagonal entry's column order
    bad.col[0], bad.col[1] = bad.col[1], bad.col[0]
    keep, As = _args(amg, systems + [(bad, None)])
    with pytest.raises(amg.AmgError) as e:
        amg.amg_setup_batch(As, None, gpu_params(amg, **KW))
    assert e.value.status == amg.AMG_ERR_INVALID_ARG and "system 3" in str(e.value)


def test_empty_batch(amg):
    st, infos = amg.amg_solve_batch([], [], [], 1e-8)
    assert st == 0 and infos == []


def test_shared_hierarchy_many_right_hand_sides(amg, oracle_lib):
    # one hierarchy serving several right-hand sides (the batch refers to it, copies nothing)
    systems = _systems()[:2]
    hs = _setup(amg, systems, **KW)
    A0, A1 = systems[0][0], systems[1][0]
    bs = [P.rhs_uniform(A0.n, 11), P.rhs_uniform(A0.n, 12), systems[1][1], P.rhs_uniform(A0.n, 13)]
    handles = [hs[0], hs[0], hs[1], hs[0]]
    mats = [A0, A0, A1, A0]
    xs = [np.zeros(len(b)) for b in bs]
    st, infos = amg.amg_solve_batch(handles, bs, xs, 1e-8)
    assert st == 0
    for h, A, b, x, info in zip(handles, mats, bs, xs, infos):
        xa = np.zeros(len(b))
        ia = amg.amg_solve(h, b, xa, 1e-8)
        assert info.status == 0
        assert iterations_agree(oracle_lib, A, KW, b, 1e-8, info.iters, ia.iters), (info.iters, ia.iters)
        assert np.linalg.norm(x - xa) / np.linalg.norm(xa) <= SOL_TOL
    for h in hs:
        amg.amg_free(h)


def test_tuned_batch_and_repeated_solves(amg):
    # lanes per row picked by timing; a second solve with the same batch reuses its graphs
    systems = _systems()
    hs = _setup(amg, systems, precision=1, **KW)
    bt = amg.amg_batch_create(hs, tune=True)
    bs = [b for _, b in systems]
    x1 = [np.zeros(A.n) for A, _ in systems]
    x2 = [np.zeros(A.n) for A, _ in systems]
    st1, i1 = amg.amg_batch_solve(bt, bs, x1, 1e-8)
    st2, i2 = amg.amg_batch_solve(bt, bs, x2, 1e-8)
    amg.amg_batch_free(bt)
    assert st1 == 0 and st2 == 0
    for k, (A, b) in enumerate(systems):
        assert i1[k].iters == i2[k].iters and np.array_equal(x1[k], x2[k])
        xa = np.zeros(A.n)
        ia = amg.amg_solve(hs[k], b, xa, 1e-8)
        assert abs(i1[k].iters - ia.iters) <= 1
        assert np.linalg.norm(x1[k] - xa) / np.linalg.norm(xa) <= 1e-6
    for h in hs:
        amg.amg_free(h)
