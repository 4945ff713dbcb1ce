"""The bench's multi-rank path on the CPU: two gloo ranks (one process per
GPU on a GPU machine) agree on the slowest rank's time, and the whole-job rate
counts every rank's work (replicas, weak scaling)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, times, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    ms = bench.max_over_ranks(times[rank], dist, torch.device("cpu"))
    rate = bench.whole_job_rate(world, 1000, ms)
    out.put((rank, ms, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [12.5, 40.0]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in res:
        assert ms == 40.0
        assert rate == pytest.approx(2 * 1000 / 0.040)


def test_single_process_is_unchanged():
    import bench
    assert bench.max_over_ranks(7.0, None, None) == 7.0
    assert bench.whole_job_rate(1, 500, 250.0) == pytest.approx(2000.0)
