"""The multi-rank path of bench.py on CPU: N ranks run N independent
replicas, and the line reports their summed work over the slowest rank's
time.  Two gloo ranks check combine_ranks (max of the times, sum of the
work) and the replica seeds (seed + rank give distinct initial states)."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_1407_7105_gb300 import ics


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        maxes, sums = bench.combine_ranks([1.5 + rank, 2.0 - rank], [10.0 * (rank + 1), 0.25], "cpu")
        m, x, _ = ics.plummer(64, seed=1 + rank)
        out[rank] = (maxes, sums, float(x[0, 0]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        maxes, sums, _ = res[r]
        assert maxes == [2.5, 2.0] and sums == [30.0, 0.5]
    assert res[0][2] != res[1][2]  # replicas start from different states


def test_single_process_passthrough():
    assert bench.combine_ranks([1.0, 2.0], [3.0], "cpu") == ([1.0, 2.0], [3.0])
