"""The sharded path on CPU (world_size-2 gloo ranks): the row partition of one
batch, and the single all-reduce of the variational step.  The per-rank
numbers come from the FP64 oracle (the GPU path is the same per pair).

* The partition covers every row exactly once in contiguous ranges with about
  equal pair counts, also for ragged and empty rows.
* Per-pair outputs computed on each rank's share equal, bit for bit, those of
  the whole batch computed at once (the pairs are independent).
* Each rank sums the Gaussian log-likelihood and its gradient over its share
  of the supernovae for the same guide samples; after the all-reduce every
  rank holds the whole sum, equal to the single-rank sum to FP64 rounding.
"""
import os
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2212_01937_gb300 import shard, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_row_ranges_cover_and_balance():
    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 8):
        for _ in range(20):
            lens = np.floor(10 ** rng.uniform(0, 3, rng.integers(1, 200))).astype(np.int64)
            lens[rng.random(lens.size) < 0.1] = 0
            off = np.concatenate([[0], np.cumsum(lens)])
            rr = shard.row_ranges(off, world)
            assert rr[0][0] == 0 and rr[-1][1] == lens.size
            assert all(a[1] == b[0] for a, b in zip(rr, rr[1:]))
            per = [int(off[r1] - off[r0]) for r0, r1 in rr]
            assert sum(per) == off[-1]
            assert max(per) - off[-1] / world <= lens.max() + 1


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # per-pair outputs on this rank's share of a ragged batch
    b = workloads.ragged_batch(B=30, seed=3, nmax_exp=2.0)
    p, z, off, rows, pairs = shard.local_batch(b.params, b.z, b.offsets, rank, world)
    res = oracle.quad_distances(p, z, off)
    # the variational step's exchange: all samples, this rank's supernovae
    sn = workloads.supernovae(N=600, seed=1)
    S = 5
    theta = np.array([[70.0 + s, 0.3 + 0.01 * s, 0.7 - 0.01 * s, 5e-5] for s in range(S)])
    cut = shard.row_ranges(np.arange(sn.nnz + 1), world)[rank]
    zl, ml = sn.z[cut[0]:cut[1]], sn.m_obs[cut[0]:cut[1]]
    ll = np.zeros(S)
    g = np.zeros((S, 4))
    for s in range(S):
        o, J = oracle.quad_distances(theta[s:s + 1], zl, np.array([0, zl.size]), grad=True)
        r = (ml - o[:, 5] - sn.M) / sn.sigma
        ll[s] = np.sum(-0.5 * r * r - np.log(sn.sigma * np.sqrt(2 * np.pi)))
        g[s] = ((r / sn.sigma)[:, None] * J[:, 5, :]).sum(axis=0)
    llt, gt = torch.tensor(ll), torch.tensor(g)
    shard.allreduce_loglike(llt, gt)
    out[rank] = (rows, pairs, res, llt.numpy(), gt.numpy())
    dist.destroy_process_group()


def test_two_gloo_ranks_partition_and_allreduce():
    port = 29600 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    b = workloads.ragged_batch(B=30, seed=3, nmax_exp=2.0)
    whole = oracle.quad_distances(b.params, b.z, b.offsets)
    got = np.zeros_like(whole)
    for r in (0, 1):
        _, (p0, p1), part, _, _ = res[r]
        got[p0:p1] = part
    assert res[0][1][1] == res[1][1][0] and res[1][1][1] == b.nnz
    assert np.array_equal(got, whole)
    # the all-reduced sums: equal on both ranks, and equal to one rank's sum
    sn = workloads.supernovae(N=600, seed=1)
    S = 5
    theta = np.array([[70.0 + s, 0.3 + 0.01 * s, 0.7 - 0.01 * s, 5e-5] for s in range(S)])
    ll = np.zeros(S)
    g = np.zeros((S, 4))
    for s in range(S):
        o, J = oracle.quad_distances(theta[s:s + 1], sn.z, np.array([0, sn.nnz]), grad=True)
        rr = (sn.m_obs - o[:, 5] - sn.M) / sn.sigma
        ll[s] = np.sum(-0.5 * rr * rr - np.log(sn.sigma * np.sqrt(2 * np.pi)))
        g[s] = ((rr / sn.sigma)[:, None] * J[:, 5, :]).sum(axis=0)
    assert np.array_equal(res[0][3], res[1][3]) and np.array_equal(res[0][4], res[1][4])
    assert np.allclose(res[0][3], ll, rtol=1e-13, atol=0)
    assert np.allclose(res[0][4], g, rtol=1e-12, atol=1e-12 * np.abs(g).max())
