"""The multi-rank path of the benchmark on CPU ranks (gloo, world size 2).

Each rank solves its own cell (own microstructure seed) with no data
exchange; the job's time is the slowest rank's and its work the sum over
ranks. This checks that reduction and the per-rank seeds without a GPU.
"""
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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dev_ms = 100.0 + 50.0 * rank
    wall_ms = 120.0 + 10.0 * rank
    units = 1000.0 * (rank + 1)
    launches = 7 + rank
    res = bench.reduce_over_ranks(dist, dev_ms, wall_ms, units, launches, "cpu")
    out[rank] = (res, bench.rank_seed(rank))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        (dev, wall, units, launches), seed = out[r]
        assert dev == 150.0 and wall == 130.0          # slowest rank
        assert units == 3000.0 and launches == 15       # sum over ranks
    assert out[0][1] != out[1][1]                       # own microstructure per rank
