"""Host logic of the multi-rank bench path on CPU: two gloo ranks, the job
time is the maximum over ranks and the rate counts the units of all ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], world)
        out[rank] = (t, bench.whole_job_rate(10, world, t))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    times = [120.0, 80.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, times, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(100)
        assert p.exitcode == 0
    for r in range(world):
        t, rate = out[r]
        assert t == 120.0
        assert abs(rate - 2 * 10 / 0.12) < 1e-9


def test_single_rank_is_identity():
    assert bench.max_over_ranks(42.0, 1) == 42.0
    assert bench.whole_job_rate(5, 1, 500.0) == 10.0
