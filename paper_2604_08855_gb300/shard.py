"""Sharding of the primaries over ranks (one process per GPU).

zeta is a sum over primaries, so ranks can own disjoint primary sets, keep
every point as a secondary, and combine their partial zeta with one float64
all-reduce of (l_max+1) * nbins^2 values (the only exchange step).  The
partition is contiguous in a seeded permutation, so every rank derives the
same split without communication.
"""
from __future__ import annotations

import numpy as np


def shard_primaries(n: int, rank: int, world: int, seed: int = 0) -> np.ndarray:
    """Primary indices owned by `rank` (sorted); the shards partition range(n)."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    perm = np.random.default_rng(seed).permutation(n)
    lo = (n * rank) // world
    hi = (n * (rank + 1)) // world
    return np.sort(perm[lo:hi]).astype(np.int64)


def allreduce_zeta(zeta_part: np.ndarray, group=None) -> np.ndarray:
    """Sum the ranks' partial zeta in float64 (torch.distributed, any backend)."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(zeta_part, dtype=np.float64))
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


def sharded_zeta(est, rank: int, world: int, seed: int = 0, group=None) -> np.ndarray:
    """zeta over all primaries from this rank's shard plus the all-reduce.

    `est` is a ctb.CTB holding the full catalogue (every point is a secondary).
    """
    prim = shard_primaries(est.n, rank, world, seed)
    return allreduce_zeta(est.compute_subset(prim), group)
