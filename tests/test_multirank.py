"""The benchmark's multi-rank path on the CPU: two gloo ranks, each with its
own shard, the slowest rank's time, and the whole-job value."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2202_10647_gb300 import workloads as W


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank: int, world: int, port: int, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = W.nitrogen_3d(2, 4, 8, seed=bench.shard_seed(rank))
        # a rank-dependent "time": the reduction must return the largest
        total_ms = 10.0 + 5.0 * rank
        worst = bench.max_over_ranks(total_ms, dist, torch.device("cpu"))
        dist.barrier()
        value = bench.job_value(world, wl.ncells, 3, worst)
        # each rank's shard checksum, gathered to compare
        chk = torch.tensor([float(wl.E.double().sum())], dtype=torch.float64)
        got = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(got, chk)
        out[rank] = (worst, value, [float(g) for g in got])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    n = 2 * 4 * 8
    for r in range(world):
        worst, value, sums = res[r]
        assert worst == 15.0                             # the slowest rank
        assert value == pytest.approx(world * n * 3 / 15e-3)
        assert sums[0] != sums[1]                        # shards differ
    assert res[0][2] == res[1][2]
