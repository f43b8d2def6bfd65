"""The N > 1 bench path on CPU: world-size-2 gloo ranks each 'step' their own replica;
the job's time is the max over ranks and the value counts every rank's units (replicas
only: no collective in the data path)."""
import os
import socket

import pytest
import torch
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        mine = [10.0 + rank, 5.0 * (2 - rank), 3.0]           # per-rank timings (ms)
        agg = bench.max_over_ranks(mine, world, "cpu")
        val = bench.job_throughput(1000.0, world, agg[0])
        q.put((rank, agg, val))
    finally:
        dist.destroy_process_group()


def test_replicas_max_over_ranks_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, agg, val in out:
        assert agg == [11.0, 10.0, 3.0]                          # the slowest rank per entry
        assert val == pytest.approx(1000.0 * 2 / 11e-3)          # both ranks' units / max time


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]
    assert bench.job_throughput(100.0, 1, 10.0) == pytest.approx(1e4)
