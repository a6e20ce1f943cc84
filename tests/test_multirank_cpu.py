"""The benchmark's multi-rank aggregation (one process per GPU, replicas): the slowest rank's
time and the whole-job throughput, checked with two gloo processes on the CPU."""
from __future__ import annotations

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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units, ms = 1000.0 * (rank + 1), 10.0 * (rank + 1)
    value, slowest = bench.aggregate_ranks(units, ms, world, torch.device("cpu"))
    out[rank] = (value, slowest)
    dist.destroy_process_group()


def test_two_rank_aggregation_takes_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # every rank reports the same slowest time (20 ms) and value = units per rank x ranks / slowest
    for r in range(world):
        value, slowest = res[r]
        assert slowest == pytest.approx(20.0)
        assert value == pytest.approx((1000.0 * (r + 1)) * world / 0.020)
