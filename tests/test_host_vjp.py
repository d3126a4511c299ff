"""lcdm_distances_vjp_host (host arrays, chunked copies overlapping the
kernels) gives the results of lcdm_distances_vjp on device arrays: the same
per-pair outputs and the same per-cosmology gradients (FP64 sums, summation
order aside), for ragged rows with empty ones, any chunk count, and when
called twice in a row with the same buffers."""
import numpy as np
import pytest
import torch

from paper_2212_01937_gb300 import workloads

pytestmark = pytest.mark.gpu
OUTS = ("d_C", "t", "X", "mu")


def _ragged(seed=3):
    b = workloads.ragged_batch(B=40, seed=seed, nmax_exp=2.5)
    return b


@pytest.mark.parametrize("nchunks", [1, 3, 64])
def test_host_entry_matches_device_entry(lib, nchunks):
    b = _ragged()
    dev = torch.device("cuda:0")
    g = torch.Generator().manual_seed(5)
    cot = {o: torch.randn(b.nnz, generator=g, dtype=torch.float32) for o in OUTS}
    p_h = torch.tensor(b.params).contiguous()
    z_h = torch.tensor(b.z, dtype=torch.float32).pin_memory()
    off_h = torch.tensor(b.offsets)
    cot_h = {o: v.pin_memory() for o, v in cot.items()}
    ref = lib.distances_vjp(p_h.to(dev), z_h.to(dev), {o: v.to(dev) for o, v in cot.items()}, off_h.to(dev),
                            outputs=OUTS, precision="fp32")
    host = lib.HostVJP(b.B, b.nnz, outputs=OUTS, nchunks=nchunks)
    for _ in range(2):
        res = host(p_h, z_h, cot_h, off_h)
        torch.cuda.synchronize()
        for o in OUTS:
            assert torch.equal(res[o], ref[o].cpu()), o
        assert torch.equal(res["status"], ref["status"].cpu())
        assert torch.allclose(res["grad"], ref["grad"].cpu(), rtol=1e-12, atol=1e-12)


def test_host_entry_rejects_bad_offsets(lib):
    b = _ragged()
    host = lib.HostVJP(b.B, b.nnz, outputs=("d_C",), nchunks=2)
    off = torch.tensor(b.offsets)
    off[-1] += 1                      # does not end at n
    with pytest.raises(RuntimeError):
        host(torch.tensor(b.params), torch.tensor(b.z, dtype=torch.float32), {"d_C": torch.zeros(b.nnz)}, off)
