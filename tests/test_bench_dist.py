"""Multi-rank host logic of bench.py on CPU: two gloo ranks time different
amounts, the reported time is the slowest rank's and the rate counts the
units of every rank (replicas of the same problem)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        assert (ws, r, local) == (world, rank, rank)
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, torch.device("cpu"))
        rate = bench.whole_job_rate(1000, ws, ms)
        dist.barrier()
        out[rank] = (ms, rate)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]
    ms, rate = res[0]
    assert ms == 15.0
    assert rate == pytest.approx(2 * 1000 / 15e-3)


def test_single_rank_needs_no_group():
    assert bench.max_over_ranks(3.5, None, None) == 3.5
    assert bench.whole_job_rate(10, 1, 2.0) == pytest.approx(5000.0)
