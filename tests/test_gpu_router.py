"""The router in front of two servers (amg_router_submit / amg_router_wait).

Both servers run on the same GPU here (one GPU per test run): the routing, the per-device
hierarchy caches and the ticket handling are those of a multi-GPU process; only the devices
coincide.  Each result must be its operator solved alone (FP64: PCG iterations by the
borderline rule, solutions within SOL_TOL), and a repeated operator must find its hierarchy
on its home server (cache hit).  Servers never wait on one another, so two on one GPU is an
ordinary configuration, not a stand-in for kernels that synchronise across devices.
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


def test_router_over_two_servers(amg, oracle_lib):
    mats = [P.stretched_box(10, 1.1), P.random_coefficient_cube(9, 3, 2.0), P.stretched_box(13, 1.15),
            P.random_coefficient_cube(11, 4, 2.0)]
    args = [amg.csr_arg(A.n, A.row_ptr, A.col, A.val) for A in mats]
    p = gpu_params(amg, **KW)
    cfgs = [amg.amg_server_config_default(p, hbm_budget_bytes=4 << 30, setup_threads=2, max_systems=64,
                                          max_rows=1 << 20, tune=0) for _ in range(2)]
    servers = [amg.amg_server_create(c) for c in cfgs]
    r = amg.amg_router_create(2)
    for d, srv in enumerate(servers):
        amg.amg_router_attach(r, d, srv)
    plan = [0, 1, 2, 0, 3, 1, 2, 0, 3]
    reqs = []
    for j, o in enumerate(plan):
        b = P.rhs_uniform(mats[o].n, 700 + j)
        x = np.zeros(mats[o].n)
        t, d = amg.amg_router_submit(r, args[o], 1, b, x)
        reqs.append((o, b, x, t, d))
    results = [amg.amg_router_wait(r, t) for *_, t, _ in reqs]
    stats = [amg.amg_router_stats(r, d) for d in range(2)]
    amg.amg_router_destroy(r)
    sstats = [amg.amg_server_stats(s) for s in servers]
    for s in servers:
        amg.amg_server_destroy(s)
    home = {}
    seen = set()
    for (o, b, x, t, d), (info, served_by) in zip(reqs, results):
        assert served_by == d and home.setdefault(o, d) == d
        assert info.status == 0 and info.relres_max <= 1e-8
        assert info.cache_hit == (1 if o in seen else 0)
        seen.add(o)
        h, st = amg.amg_setup_status(args[o], None, p)
        assert st == 0
        xa = np.zeros(mats[o].n)
        ia = amg.amg_solve(h, b, xa, 1e-8)
        amg.amg_free(h)
        assert iterations_agree(oracle_lib, mats[o], KW, b, 1e-8, info.iters_max, ia.iters)
        assert np.linalg.norm(x - xa) / np.linalg.norm(xa) <= SOL_TOL
    assert {d for *_, d in reqs} == {0, 1}
    assert [s["requests"] for s in stats] == [s.completed for s in sstats]
    assert sum(s.cache_misses for s in sstats) == len(mats)
