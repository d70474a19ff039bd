"""The benchmark's multi-rank logic (one process per GPU) on CPU: two gloo ranks
report different step times; every rank must take the slowest, and the
whole-job throughput counts the units of both ranks over that time."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [1.0 + rank, 0.25 * (2 - rank)]          # rank 1 is slower per step, rank 0 per launch
        ms, launch = bench.max_over_ranks(mine, "cpu")
        out[rank] = (ms, launch, bench.whole_job_value(1000, world, ms))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_sets_the_time_and_units_add_up():
    ctx = mp.get_context("spawn")
    world, port = 2, _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        ms, launch, value = res[r]
        assert ms == pytest.approx(2.0)
        assert launch == pytest.approx(0.5)
        assert value == pytest.approx(1000 * 2 / 2.0e-3)


def test_single_process_needs_no_group():
    assert bench.max_over_ranks([3.0, 1.5], "cpu") == [3.0, 1.5]
    assert bench.whole_job_value(10, 1, 1.0) == pytest.approx(1e4)
