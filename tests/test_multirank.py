"""The multi-rank path of the benchmark (replicas only, no data-path
collective) with gloo ranks on the CPU: the timed total is the slowest
rank's, every rank sees it, the job throughput counts every rank's units,
and the ranks' replicate shards tile the job's replicates exactly."""
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


@pytest.mark.parametrize("n_rep,world", [(256, 2), (256, 3), (256, 8), (5, 4), (1, 1), (7, 7)])
def test_replicate_shards_tile_the_job(n_rep, world):
    import bench
    ranges = [bench.shard_replicates(n_rep, r, world) for r in range(world)]
    covered = [rep for rep0, n in ranges for rep in range(rep0, rep0 + n)]
    assert covered == list(range(n_rep))
    sizes = [n for _, n in ranges]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1


def _shard_main(rank, world, port, out):
    import numpy as np
    import bench
    from paper_1605_01421_gb300 import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = W.config_batched(n_rep=5, n_nodes=40, days=6)
        rep0, n = bench.shard_replicates(w.n_rep, rank, world)
        s = W.replicate_range(w, rep0, n)
        # each rank reports the global replicates its shard holds and the
        # shard's initial state; gathered, they are the whole job's
        mine = torch.tensor([rep0, n, int(s.u0.sum())], dtype=torch.int64)
        got = [torch.zeros(3, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(got, mine)
        out[rank] = ([tuple(int(x) for x in g) for g in got],
                     int(np.asarray(w.u0).sum()), s.meta["rep_total"], s.n_rep,
                     len(s.events["event"]) == len(w.events["event"]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_hold_the_whole_job_between_them():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_shard_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    got, total_u0, rep_total, n_loc, same_events = out[0]
    assert out[1][0] == got
    assert [(a, b) for a, b, _ in got] == [(0, 2), (2, 3)]
    assert sum(c for _, _, c in got) == total_u0
    assert rep_total == 5 and n_loc == 2 and same_events
