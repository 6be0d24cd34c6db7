"""The request router across GPUs (amg_router_*), host logic on CPU: no server, no kernel.

A router gives each operator a home device when it first sees it (the device with the least
work so far) and routes every repeat there, so that repeats reach the server holding the
hierarchy.  Checked here: repeats keep their device; the decisions equal those of a plain
Python restatement of the documented rule; two processes (two `gloo` ranks) that see the same
stream make the same decisions and partition it, each operator's requests on one rank; the
key is the operator's content, not its buffers; invalid arguments are refused.
"""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

from paper_2103_10476_gb300 import problems as P

SETUP_WEIGHT = 20.0


@pytest.fixture(scope="module")
def amg():
    from paper_2103_10476_gb300 import build
    build.build()
    from paper_2103_10476_gb300 import amg as m
    return m


def _stream(seconds=1.5):
    reqs, ops = P.serving_stream(seconds, nmin=4, nmax=10)
    mats = [P.make_operator(o, engine="numpy") for o in ops]
    return reqs, mats


def _args(amg, mats):
    return [amg.csr_arg(A.n, A.row_ptr, A.col, A.val) for A in mats]


def _route_all(amg, ndev, reqs, args):
    r = amg.amg_router_create(ndev)
    out = [amg.amg_router_route(r, args[o], nrhs) for _, o, nrhs, _ in reqs]
    stats = [amg.amg_router_stats(r, d) for d in range(ndev)]
    amg.amg_router_destroy(r)
    return out, stats


def test_repeats_keep_their_device(amg):
    reqs, mats = _stream()
    args = _args(amg, mats)
    out, stats = _route_all(amg, 4, reqs, args)
    home, seen = {}, set()
    for (_, o, _, _), (d, key, rep) in zip(reqs, out):
        assert rep == (o in seen)
        seen.add(o)
        assert home.setdefault(o, d) == d
    assert sum(s["requests"] for s in stats) == len(reqs)
    assert sum(s["operators"] for s in stats) == len(mats)
    assert sum(s["repeats"] for s in stats) == len(reqs) - len(mats)
    assert len({d for d, _, _ in out}) == 4


def test_decisions_follow_the_least_work_rule(amg):
    # an independent restatement of the rule: new operator -> device with the least work
    # (lowest index on ties), work += nnz (nrhs + 20); repeat -> home, work += nnz nrhs
    reqs, mats = _stream()
    out, stats = _route_all(amg, 3, reqs, _args(amg, mats))
    work = [0.0, 0.0, 0.0]
    home = {}
    for (_, o, nrhs, _), (d, _, _) in zip(reqs, out):
        nnz = max(mats[o].nnz, 1)
        if o in home:
            want = home[o]
            work[want] += nnz * nrhs
        else:
            want = int(np.argmin(work))
            home[o] = want
            work[want] += nnz * (nrhs + SETUP_WEIGHT)
        assert d == want
    assert [s["work"] for s in stats] == pytest.approx(work, rel=0, abs=0)
    # balanced within the largest single request
    biggest = max(max(A.nnz, 1) * (8 + SETUP_WEIGHT) for A in mats)
    assert max(work) - min(work) <= biggest


def test_key_is_the_content(amg):
    A = P.stretched_box(6, 1.1)
    B = P.CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val.copy())
    C = P.CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val.copy())
    C.val[5] *= 1.0 + 2.0 ** -40
    r = amg.amg_router_create(2)
    d1, k1, rep1 = amg.amg_router_route(r, amg.csr_arg(A.n, A.row_ptr, A.col, A.val), 1)
    d2, k2, rep2 = amg.amg_router_route(r, amg.csr_arg(B.n, B.row_ptr, B.col, B.val), 1)
    d3, k3, rep3 = amg.amg_router_route(r, amg.csr_arg(C.n, C.row_ptr, C.col, C.val), 1)
    amg.amg_router_destroy(r)
    assert k1 == k2 and rep2 and d2 == d1
    assert k3 != k1 and not rep3 and d3 != d1


def test_invalid_arguments(amg):
    import ctypes as C
    r = C.c_void_p()
    assert amg.lib.amg_router_create(0, C.byref(r)) == amg.AMG_ERR_INVALID_ARG
    r = amg.amg_router_create(2)
    assert amg.lib.amg_router_stats(r, 2, None, None, None, None) == amg.AMG_ERR_INVALID_ARG
    assert amg.lib.amg_router_attach(r, -1, None) == amg.AMG_ERR_INVALID_ARG
    A = P.laplace_cube(3)
    x = np.zeros(A.n)
    b = np.ones(A.n)
    t, d = C.c_uint64(), C.c_int()
    # no server attached: refused after routing, before anything reaches a GPU
    st = amg.lib.amg_router_submit(r, C.byref(amg.csr_arg(A.n, A.row_ptr, A.col, A.val)), 1,
                                   b.ctypes.data_as(C.c_void_p), x.ctypes.data_as(C.c_void_p), C.byref(t), C.byref(d))
    assert st == amg.AMG_ERR_INVALID_ARG and "no server" in amg.amg_last_error()
    assert amg.lib.amg_router_wait(r, 12345, C.byref(amg.amg_request_info_t()), None) == amg.AMG_ERR_INVALID_ARG
    amg.amg_router_destroy(r)


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    from paper_2103_10476_gb300 import amg
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        reqs, mats = _stream(1.0)
        args = _args(amg, mats)
        r = amg.amg_router_create(world)
        decisions = [amg.amg_router_route(r, args[o], nrhs)[0] for _, o, nrhs, _ in reqs]
        amg.amg_router_destroy(r)
        mine = [k for k, d in enumerate(decisions) if d == rank]
        # the host-side gather of what each rank served (here: which requests)
        gathered = [None] * world
        dist.all_gather_object(gathered, {"rank": rank, "decisions": decisions, "served": mine})
        q.put((rank, gathered, [o for _, o, _, _ in reqs]))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_partition_a_stream():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        out = sorted(q.get(timeout=240) for _ in range(world))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
                p.join()
    assert all(p.exitcode == 0 for p in procs)
    _, gathered, op_of = out[0]
    assert gathered == out[1][1]                       # both ranks gathered the same picture
    assert gathered[0]["decisions"] == gathered[1]["decisions"]
    served = [set(g["served"]) for g in gathered]
    assert not (served[0] & served[1]) and served[0] | served[1] == set(range(len(op_of)))
    rank_of_op = {}
    for rank, s in enumerate(served):
        for k in s:
            assert rank_of_op.setdefault(op_of[k], rank) == rank   # an operator's requests on one rank
    assert served[0] and served[1]
