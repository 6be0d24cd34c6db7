"""The benchmark's multi-rank host logic on CPU (two `gloo` ranks): process-group start from the
launcher's environment, the barrier, the maximum over ranks, the whole-job rate (every rank's
units over the slowest rank's time, the replicas-only scaling), and the reference arm's rule
that only rank 0 works."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), BENCH_BACKEND="gloo")
    import torch.distributed as dist

    import bench
    try:
        w, r, local = bench.dist_init()
        bench.barrier(w)
        slowest = bench.max_over_ranks(w, 10.0 + 3.0 * r)      # per-rank step time, ms
        rate = bench.whole_job_rate(5 * 3, w, slowest)          # 5 solves a step, 3 steps a rank
        ref = bench.run_reference(None, w, r) if r != 0 else None
        bench.barrier(w)
        q.put((r, w, local, slowest, rate, ref))
    finally:
        if dist.is_initialized():
            dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks():
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
    for r, (rank, w, local, slowest, rate, ref) in enumerate(out):
        assert (rank, w, local) == (r, world, r)
        assert slowest == 13.0                     # the slower rank's time on both ranks
        assert rate == pytest.approx(15 * world / 0.013)
    assert out[1][5] == 0                          # the reference arm: rank 1 exits without work


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(1, 7.5) == 7.5
    assert bench.whole_job_rate(10, 1, 500.0) == pytest.approx(20.0)
