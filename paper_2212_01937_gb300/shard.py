"""Sharding the distance path over ranks, one GPU per rank.

The pairs are independent (Sec. 3.2.2 describes the trivial parallelisation
of the method, and fn24 its batching over cosmologies and redshifts), so:

* one batch is split into contiguous CSR row ranges with about equal pair
  counts (:func:`row_ranges`, :func:`local_batch`); per-pair outputs and
  per-row gradients need no exchange at all;
* the variational-inference step of Sec. 4 with the supernovae sharded over
  ranks (every rank evaluates all S guide samples on its share of the data)
  needs exactly one exchange: the sum over ranks of the per-sample
  log-likelihoods and their gradients, [S, 1 + ncol] FP64
  (:func:`allreduce_loglike`).  Every rank must draw the same guide samples
  (the same seed for its generator).

Only host logic and one torch.distributed all-reduce live here; the
per-rank work is the ordinary single-GPU path.
"""
import numpy as np
import torch


def row_ranges(offsets, world):
    """Contiguous row ranges [(r0, r1)] * world covering rows 0 .. B-1, cut
    at the first row that starts at or after k * nnz / world (k = 1 .. world-1),
    so that every range holds about nnz / world pairs (within one row)."""
    off = np.asarray(offsets, dtype=np.int64)
    B = off.size - 1
    nnz = int(off[-1])
    cuts = [0]
    for k in range(1, world):
        target = (nnz * k) // world
        r = int(np.searchsorted(off[:-1], target, side="left"))
        cuts.append(min(max(r, cuts[-1]), B))
    cuts.append(B)
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


def local_batch(params, z, offsets, rank, world):
    """The rank's share of a CSR batch: its parameter rows, its redshifts and
    its offsets rebased to start at 0, plus the global pair range it covers."""
    off = np.asarray(offsets, dtype=np.int64)
    r0, r1 = row_ranges(off, world)[rank]
    p0, p1 = int(off[r0]), int(off[r1])
    return params[r0:r1], z[p0:p1], off[r0:r1 + 1] - p0, (r0, r1), (p0, p1)


def allreduce_loglike(loglike, grad, group=None):
    """Sum the per-sample log-likelihoods [S] and gradients [S, ncol] (FP64)
    over the ranks of ``group`` in one all-reduce; returns them in place."""
    import torch.distributed as dist
    S = loglike.shape[0]
    buf = torch.cat([loglike.reshape(S, 1), grad], dim=1).contiguous()
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    loglike.copy_(buf[:, 0])
    grad.copy_(buf[:, 1:])
    return loglike, grad
