"""The multi-rank bench path on CPU: two gloo ranks, each with its own bins, the
job's time is the slowest rank's, and the value counts every rank's bins."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [100.0 + 50.0 * rank, 300.0 - 50.0 * rank, 7.0]
        got = bench.reduce_max(local, world, torch.device("cpu"))
        dist.barrier()
        q.put((rank, got, bench.rank_seed(rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_count():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    # every rank sees the element-wise max over ranks
    for _, got, _ in out:
        assert got == [150.0, 300.0, 7.0]
    # ranks solve different bins
    assert len({seed for _, _, seed in out}) == world
    # whole-job throughput: all ranks' units over the slowest rank's time
    assert bench.job_throughput(10, world, 150.0) == pytest.approx(2 * 10 / 0.150)


def test_single_rank_is_identity():
    assert bench.reduce_max([1.0, 2.5], 1, None) == [1.0, 2.5]
    assert bench.job_throughput(10, 1, 1000.0) == pytest.approx(10.0)
