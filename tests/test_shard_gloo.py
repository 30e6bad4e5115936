"""The multi-rank split of a batch, run as two gloo ranks on the CPU: every
instance goes to exactly one rank, the ranks agree on the split, and the
summed cost per rank is balanced."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2208_09822_gb300 import shard
from paper_2208_09822_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = W.uneven(count=20000)   # every rank draws the same batch (same seed)
    cost = shard.instance_cost(b.M, b.N, b.K, b.beta != 0)
    lo, hi = shard.shard_bounds(cost, world)[rank]
    mine = torch.tensor([lo, hi, float(cost[lo:hi].sum()), float(b.flops())], dtype=torch.float64)
    allv = [torch.zeros(4, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(allv, mine)
    if rank == 0:
        out.put([v.tolist() for v in allv])
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_cover_the_batch():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, q), nprocs=world, start_method="spawn", join=True)
    rows = q.get()
    bounds = [(int(r[0]), int(r[1])) for r in rows]
    assert bounds[0][0] == 0 and bounds[-1][1] == 20000
    for (a0, a1), (b0, b1) in zip(bounds, bounds[1:]):
        assert a1 == b0
    costs = [r[2] for r in rows]
    assert max(costs) / (sum(costs) / world) < 1.02
    assert rows[0][3] == rows[1][3]   # both ranks drew the same batch


def test_shard_bounds_edge_cases():
    assert shard.shard_bounds([], 3) == [(0, 0)] * 3
    assert shard.shard_bounds([5.0], 2) in ([(0, 0), (0, 1)], [(0, 1), (1, 1)])
    b = shard.shard_bounds(np.ones(10), 4)
    assert b[0][0] == 0 and b[-1][1] == 10
    assert sum(e - s for s, e in b) == 10
    with pytest.raises(ValueError):
        shard.shard_bounds([1.0], 0)
