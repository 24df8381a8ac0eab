"""The multi-GPU host logic of bench.py on CPU: two gloo ranks.

Events are independent problems, so ranks share no data: each draws its own
events (distinct seeds), and the only collective is the max over ranks of the
timed regions, from which the whole-job rate is formed (weak scaling).
"""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank-local timings of two regions (device-resident, end to end)
        got = bench.combine_ranks(dist, (10.0 + rank, 20.0 - rank), torch.device("cpu"))
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.rank_seed(2, rank))
        out[rank] = (got, seeds)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_by_max():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        got, seeds = res[r]
        assert got == [11.0, 20.0]          # each region: the slowest rank
        assert len(set(seeds)) == world      # independent events per rank
    # whole-job rate: every rank's units over the max-over-ranks time
    assert bench.whole_job_rate(world, 1000, 10, 11.0) == pytest.approx(2 * 1000 * 10 / 0.011)


def test_single_process_needs_no_collective():
    assert bench.combine_ranks(None, (3.0, 4.0), None) == [3.0, 4.0]


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup, gpus = 1, 1, 2
    assert bench.run_reference(A()) is None
