"""Split a batch of independent GEMM instances across ranks.

Instances share nothing, so the multi-GPU form of the grouped launch is one
plan per GPU over a contiguous shard of the instance list, with no collective
on the data path.  Shards are cut on the prefix sum of a per-instance cost
estimate so that every rank gets about the same work.
"""
from __future__ import annotations

import numpy as np


def instance_cost(M, N, K, beta_nonzero, esize=4, bytes_per_flop=0.5):
    """Cost estimate of an instance: its algorithmic bytes plus a flop term
    (HBM-bound kernels are charged mostly by bytes)."""
    M = np.asarray(M, np.float64); N = np.asarray(N, np.float64); K = np.asarray(K, np.float64)
    elems = M * K + K * N + M * N + np.where(np.asarray(beta_nonzero), M * N, 0)
    return esize * elems + bytes_per_flop * 2 * M * N * K + 64.0   # + descriptor


def shard_bounds(cost, world):
    """Contiguous [begin, end) instance ranges, one per rank, with nearly
    equal summed cost.  Every instance lands in exactly one shard."""
    cost = np.asarray(cost, np.float64)
    n = len(cost)
    if world <= 0:
        raise ValueError("world must be positive")
    if n == 0:
        return [(0, 0)] * world
    pref = np.concatenate([[0.0], np.cumsum(cost)])
    total = pref[-1]
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        c = int(np.searchsorted(pref, target, side="left"))
        c = min(max(c, cuts[-1]), n)
        cuts.append(c)
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]
