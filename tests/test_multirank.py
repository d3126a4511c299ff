"""The multi-rank path of bench.py on CPU: world_size-2 gloo ranks, each with
its own (weak-scaling) batch and step time; the job's step time is the max
over ranks and its rate counts every rank's pairs.  Each rank also draws its
own synthetic batch (seed offset by the rank)."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [2.0, 3.5][rank]
    got_ms, value = bench.aggregate(ms, 1000, world, dist, torch.device("cpu"))
    b = bench.workload(seed_offset=rank)
    out[rank] = (got_ms, value, float(b.params[0, 1]))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        got_ms, value, _ = res[r]
        assert got_ms == 3.5
        assert value == pytest.approx(2 * 1000 / 3.5e-3)
    assert res[0][2] != res[1][2]          # each rank owns a batch of its own
