"""The multi-rank path of the benchmark (replicas only: one independent
replica per rank, no data-path collective) with two gloo ranks on the CPU:
the timed total is the slowest rank's, every rank sees it, and the job
throughput counts every rank's units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 100.0 + 25.0 * rank           # the ranks' own timed totals
        got = bench.max_over_ranks(mine, dist, "cpu")
        out[rank] = (got, bench.job_throughput(584_000, 5, world, got))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 125.0
    # 2 ranks x 5 steps x 584,000 node-days in 125 ms
    assert out[0][1] == pytest.approx(2 * 5 * 584_000 / 0.125)


def test_single_process_is_the_identity():
    import bench
    assert bench.max_over_ranks(42.5, None, "cpu") == 42.5
    assert bench.job_throughput(1000, 2, 1, 1000.0) == pytest.approx(2000.0)
