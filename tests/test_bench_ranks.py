"""The multi-rank host logic of bench.py on CPU: two gloo ranks (replicas)
agree on the slowest rank's timings, and the whole-job rate counts every
rank's units over that time."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank 0 is slower in the first entry, rank 1 in the second
        got = bench.max_over_ranks([10.0 - rank, 3.0 + rank], world)
        out[rank] = torch.tensor(got)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_timing():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        assert out[r].tolist() == [10.0, 4.0]


def test_single_rank_is_identity_and_job_rate():
    import bench
    assert bench.max_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]
    # 2 replicas x 1000 units x 10 steps in 0.5 s
    assert bench.job_rate(2, 1000, 10, 500.0) == pytest.approx(40000.0)
