"""The request server (amg_server_*): continuous batching of served solves.

Each request's solutions must be those of its operator solved alone with amg_solve on a
hierarchy built with the same parameters: iteration counts within the borderline rule
(summation orders differ), solutions within SOL_TOL (FP64) or 1e-6 (mixed precision, whose
result depends on the FP32 rounding of the V-cycle).  The same request gives the same
answer alone and in a mix of other requests that arrive while it runs.
"""
import time

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


class Op:
    def __init__(self, amg, A):
        self.A = A
        self.rp = np.ascontiguousarray(A.row_ptr, np.int64)
        self.ci = np.ascontiguousarray(A.col, np.int32)
        self.v = np.ascontiguousarray(A.val, np.float64)
        self.arg = amg.csr_arg(A.n, self.rp, self.ci, self.v)


def _server(amg, precision=0, **kw):
    p = gpu_params(amg, precision=precision, **KW)
    cfg = amg.amg_server_config_default(p, hbm_budget_bytes=kw.pop("budget", 8 << 30), setup_threads=4,
                                        max_systems=kw.pop("max_systems", 256), max_rows=kw.pop("max_rows", 1 << 21),
                                        tune=0, **kw)
    return amg.amg_server_create(cfg)


def _alone(amg, op, b, precision):
    h, st = amg_setup_status(amg, op, precision)
    x = np.zeros(op.A.n)
    info = amg.amg_solve(h, b, x, 1e-8)
    amg.amg_free(h)
    return info, x


def amg_setup_status(amg, op, precision):
    h, st = amg.amg_setup_status(op.arg, None, gpu_params(amg, precision=precision, **KW))
    assert st == 0
    return h, st


def _check(amg, oracle_lib, op, b, x, info_iters, precision):
    ia, xa = _alone(amg, op, b, precision)
    if precision:
        assert abs(info_iters - ia.iters) <= 1, (info_iters, ia.iters)
    else:
        assert iterations_agree(oracle_lib, op.A, KW, b, 1e-8, info_iters, ia.iters), (info_iters, ia.iters)
    assert np.linalg.norm(x - xa) / np.linalg.norm(xa) <= (1e-6 if precision else SOL_TOL)


@pytest.mark.parametrize("precision", [0, 1])
def test_served_requests_equal_solves_alone(amg, oracle_lib, precision):
    ops = [Op(amg, A) for A in (P.stretched_box(12, 1.1), P.random_coefficient_cube(10, 3, 2.0),
                                P.stretched_box(15, 1.2), P.laplace_cube(7))]
    srv = _server(amg, precision)
    # requests: (operator, number of right-hand sides); operators repeat
    plan = [(0, 1), (1, 3), (0, 2), (2, 1), (3, 2), (1, 1), (2, 2), (0, 1)]
    reqs = []
    for j, (o, nrhs) in enumerate(plan):
        n = ops[o].A.n
        b = np.concatenate([P.rhs_uniform(n, 100 * j + k) for k in range(nrhs)])
        x = np.zeros(nrhs * n)
        t = amg.amg_server_submit(srv, ops[o].arg, nrhs, b, x)
        reqs.append((o, nrhs, b, x, t))
    infos = [amg.amg_server_wait(srv, t) for *_, t in reqs]
    stats = amg.amg_server_stats(srv)
    amg.amg_server_destroy(srv)
    assert stats.completed == len(plan) and stats.solves == sum(n for _, n in plan)
    assert stats.cache_misses == len(ops) and stats.cache_hits == len(plan) - len(ops)
    for (o, nrhs, b, x, _), info in zip(reqs, infos):
        assert info.status == 0 and info.relres_max <= 1e-8 and info.nrhs == nrhs
        n = ops[o].A.n
        alone = []
        for k in range(nrhs):
            ia, xa = _alone(amg, ops[o], b[k * n:(k + 1) * n], precision)
            assert np.linalg.norm(x[k * n:(k + 1) * n] - xa) / np.linalg.norm(xa) <= (1e-6 if precision else SOL_TOL)
            alone.append(ia.iters)
        # the request reports the most iterations any of its right-hand sides took
        k = int(np.argmax(alone))
        if precision:
            assert abs(info.iters_max - alone[k]) <= 1, (info.iters_max, alone)
        else:
            assert iterations_agree(oracle_lib, ops[o].A, KW, b[k * n:(k + 1) * n], 1e-8, info.iters_max,
                                    alone[k]), (info.iters_max, alone)


def test_same_result_alone_and_in_a_mix(amg, oracle_lib):
    # the request alone on an idle server, then the same request submitted while a large,
    # slow request runs and others keep arriving
    target = Op(amg, P.random_coefficient_cube(11, 5, 2.0))
    big = Op(amg, P.stretched_box(28, 1.15))
    others = [Op(amg, P.stretched_box(10 + k, 1.1)) for k in range(4)]
    b = P.rhs_uniform(target.A.n, 7)
    srv = _server(amg, 0)
    x_alone = np.zeros(target.A.n)
    i_alone = amg.amg_server_wait(srv, amg.amg_server_submit(srv, target.arg, 1, b, x_alone))
    xb = np.zeros(big.A.n)
    tb = amg.amg_server_submit(srv, big.arg, 1, P.rhs_uniform(big.A.n, 1), xb)
    time.sleep(0.05)
    keep = []
    ts = []
    for k, op in enumerate(others):
        bo = P.rhs_uniform(op.A.n, 50 + k)
        xo = np.zeros(op.A.n)
        keep.append((bo, xo))
        ts.append(amg.amg_server_submit(srv, op.arg, 1, bo, xo))
    x_mix = np.zeros(target.A.n)
    tt = amg.amg_server_submit(srv, target.arg, 1, b, x_mix)
    i_mix = amg.amg_server_wait(srv, tt)
    for t in ts:
        assert amg.amg_server_wait(srv, t).status == 0
    ib = amg.amg_server_wait(srv, tb)
    amg.amg_server_destroy(srv)
    assert i_alone.status == 0 and i_mix.status == 0 and ib.status == 0
    assert i_mix.cache_hit == 1
    # lanes chosen by row length (tune = 0): a member's arithmetic does not depend on the others
    assert i_mix.iters_max == i_alone.iters_max
    assert np.linalg.norm(x_mix - x_alone) / np.linalg.norm(x_alone) <= SOL_TOL
    _check(amg, oracle_lib, target, b, x_mix, i_mix.iters_max, 0)


def _engine_bytes(amg, **kw):
    srv = _server(amg, 0, **kw)
    b = amg.amg_server_stats(srv).bytes_engine
    amg.amg_server_destroy(srv)
    return b


def _estimate(A):
    return 64 * A.nnz + 160 * A.n + (1 << 20)


def test_eviction_under_a_small_budget(amg, oracle_lib):
    ops = [Op(amg, P.stretched_box(14 + k, 1.1)) for k in range(5)]
    small = dict(max_rows=1 << 18, max_systems=16)
    budget = _engine_bytes(amg, **small) + 3 * _estimate(ops[-1].A) // 2
    srv = _server(amg, 0, budget=budget, **small)
    out = []
    for k, op in enumerate(ops + ops[:2]):
        b = P.rhs_uniform(op.A.n, k)
        x = np.zeros(op.A.n)
        info = amg.amg_server_wait(srv, amg.amg_server_submit(srv, op.arg, 1, b, x))
        out.append((op, b, x, info))
    stats = amg.amg_server_stats(srv)
    amg.amg_server_destroy(srv)
    assert stats.evictions > 0 and stats.resident_hierarchies < len(ops)
    assert stats.bytes_hierarchies + stats.bytes_engine <= budget
    for op, b, x, info in out:
        assert info.status == 0
        _check(amg, oracle_lib, op, b, x, info.iters_max, 0)


def test_request_larger_than_budget_fails(amg):
    small = dict(max_rows=1 << 17, max_systems=8)
    op = Op(amg, P.stretched_box(40, 1.1))
    srv = _server(amg, 0, budget=_engine_bytes(amg, **small) + _estimate(op.A) // 2, **small)
    x = np.zeros(op.A.n)
    info = amg.amg_server_wait(srv, amg.amg_server_submit(srv, op.arg, 1, P.rhs_uniform(op.A.n, 1), x))
    amg.amg_server_destroy(srv)
    assert info.status == amg.AMG_ERR_BUDGET


def test_zero_rhs_requests_and_poll(amg):
    op = Op(amg, P.stretched_box(9, 1.1))
    srv = _server(amg, 0)
    t0 = amg.amg_server_submit(srv, op.arg, 0, None, None)
    b = np.zeros(2 * op.A.n)
    x = np.full(2 * op.A.n, 3.0)
    t1 = amg.amg_server_submit(srv, op.arg, 2, b, x)
    info0 = amg.amg_server_wait(srv, t0)
    for _ in range(2000):
        info1 = amg.amg_server_poll(srv, t1)
        if info1 is not None:
            break
        time.sleep(0.005)
    amg.amg_server_destroy(srv)
    assert info0.status == 0 and info0.nrhs == 0
    assert info1 is not None and info1.status == 0 and info1.iters_max == 0 and not x.any()


@pytest.mark.parametrize("precision", [0, 1])
def test_served_results_match_oracle(amg, oracle_lib, precision):
    # served results against the oracle directly: FP64 by the borderline rule and within SOL_TOL,
    # mixed precision within one iteration of the FP64 oracle and 1e-6 of its solution
    ops = [Op(amg, A) for A in (P.stretched_box(13, 1.12), P.random_coefficient_cube(12, 4, 2.0))]
    srv = _server(amg, precision)
    reqs = []
    for j, op in enumerate(ops + ops[:1]):
        b = P.rhs_uniform(op.A.n, 300 + j)
        x = np.zeros(op.A.n)
        reqs.append((op, b, x, amg.amg_server_submit(srv, op.arg, 1, b, x)))
    infos = [amg.amg_server_wait(srv, t) for *_, t in reqs]
    amg.amg_server_destroy(srv)
    for (op, b, x, _), info in zip(reqs, infos):
        assert info.status == 0 and info.relres_max <= 1e-8
        oh, ost = oracle_lib.setup(op.A, **KW)
        assert ost == 0
        xo, oinfo, _ = oh.solve(b, 1e-8)
        if precision:
            assert abs(info.iters_max - oinfo.iters) <= 1, (info.iters_max, oinfo.iters)
            assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-6
        else:
            assert iterations_agree(oracle_lib, op.A, KW, b, 1e-8, info.iters_max, oinfo.iters)
            assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= SOL_TOL
