"""Multi-rank decomposition of zeta over primaries: world size 2, gloo, CPU.

Each rank runs shard.sharded_zeta itself -- the product's multi-GPU step:
its shard of the primaries, compute_subset over that shard, then the float64
all-reduce -- with an estimator stand-in whose compute_subset is the FP64
oracle (no GPU here).  The test checks that every rank ends with the full
zeta and that the shards partition the primaries.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2604_08855_gb300 import shard, synth

KW = dict(box=200.0, rmin=2.0, rmax=30.0, nbins=4, lmax=4)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleEstimator:
    """Stands in for ctb.CTB in sharded_zeta: the same n / compute_subset
    interface, computed by the FP64 oracle; records the primaries it got."""

    def __init__(self, xyz, w, kw):
        self.xyz, self.w, self.kw = xyz, w, kw
        self.n = xyz.shape[0]
        self.seen = None

    def compute_subset(self, prim):
        import oracle
        self.seen = np.asarray(prim)
        return oracle.zeta(self.xyz, self.w, prim=self.seen, nthreads=1, **self.kw)["zeta"]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    xyz, w = synth.thomas(1500, 200.0, 15, 4.0, seed=31, weights="u0.5-1.5")
    est = OracleEstimator(xyz, w, KW)
    total = shard.sharded_zeta(est, rank, world, seed=5)
    np.save(os.path.join(out, f"z{rank}.npy"), total)
    np.save(os.path.join(out, f"p{rank}.npy"), est.seen)
    dist.destroy_process_group()


def test_shards_partition():
    for world in (1, 2, 3, 7):
        parts = [shard.shard_primaries(1000, r, world, seed=2) for r in range(world)]
        allp = np.concatenate(parts)
        assert np.array_equal(np.sort(allp), np.arange(1000))


def test_two_rank_allreduce_matches_full(tmp_path):
    import oracle
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    xyz, w = synth.thomas(1500, 200.0, 15, 4.0, seed=31, weights="u0.5-1.5")
    full = oracle.zeta(xyz, w, **KW)["zeta"]
    z0 = np.load(tmp_path / "z0.npy")
    z1 = np.load(tmp_path / "z1.npy")
    assert np.array_equal(z0, z1)
    assert np.allclose(z0, full, rtol=1e-12, atol=1e-12 * np.abs(full).max())
    p0, p1 = np.load(tmp_path / "p0.npy"), np.load(tmp_path / "p1.npy")
    assert np.intersect1d(p0, p1).size == 0 and p0.size + p1.size == xyz.shape[0]
    assert np.array_equal(p0, shard.shard_primaries(xyz.shape[0], 0, world, seed=5))
