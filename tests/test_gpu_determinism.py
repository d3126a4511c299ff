"""The opt-in deterministic reduction (lcdm_opts.deterministic): the
per-cosmology sums of the fused adjoint and of the log-likelihood give the
same bits on repeated calls with the same inputs and launch shape, and agree
with the default (atomic) reduction to FP64 rounding.  Short rows make many
rows shared between the persistent warps' pair ranges."""
import numpy as np
import pytest
import torch

from paper_2212_01937_gb300 import workloads
from test_gpu_parity import DEV, _t

pytestmark = pytest.mark.gpu


def _batch():
    b = workloads.ragged_batch(B=3000, seed=5, nmax_exp=2.2)
    return b


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_vjp_and_loglike_reproducible(lib, prec):
    b = _batch()
    dt = np.float64 if prec == "fp64" else np.float32
    p, off = _t(b.params), _t(b.offsets)
    z, m = _t(b.z.astype(dt)), _t(b.m_obs.astype(dt))
    rng = np.random.default_rng(3)
    cot = {n: _t(rng.normal(size=b.nnz).astype(dt)) for n in ("d_C", "t", "mu")}
    runs = []
    for det in (True, True, False):
        call = lib.Call(p, z, off, precision=prec, block=128, blocks_per_sm=2, lane_map="contiguous",
                        deterministic=det)
        g = lib.distances_vjp(p, z, cot, off, outputs=("d_C",), call=call)["grad"].clone()
        ll = lib.gauss_loglike(p, z, m, off, M=b.M, sigma=b.sigma, call=call)
        runs.append((g, ll["loglike"].clone(), ll["grad"].clone()))
    torch.cuda.synchronize()
    for a, c in zip(runs[0], runs[1]):
        assert torch.equal(a, c)
    for a, c in zip(runs[0], runs[2]):
        assert torch.allclose(a, c, rtol=1e-12, atol=1e-9 * float(c.abs().max()), equal_nan=True)
