"""Seven-column rows (the further components of fn4, w = -1/3 and -2/3):
forward distances and the magnitude log-likelihood through the C ABI against
the oracle; tangent-requiring calls are refused.  Tolerances as for the
five-column path (test_gpu_parity.py)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_01937_gb300 import workloads

from test_gpu_parity import TOL32, TOL64, _check, _t

pytestmark = pytest.mark.gpu

ALL = ("d_C", "t", "X", "d_M", "d_L", "mu")


def _rows():
    """Mixtures with radiation (quartic) and without (cubic); 37 redshifts
    per row over U(0, 10) with 1e-3 and 1100 planted."""
    P = np.array([[70.0, 0.3, 0.6, 5e-5, 0.05, 0.03, 0.02 - 5e-5],
                  [68.0, 0.25, 0.5, 8e-5, -0.05, 0.2, 0.1 - 8e-5],
                  [72.0, 0.4, 0.7, 3e-5, 0.0, -0.05, -0.05 - 3e-5],
                  [70.0, 0.3, 0.6, 0.0, 0.0, 0.05, 0.05],
                  [66.0, 0.2, 0.8, 0.0, -0.1, 0.08, 0.02]])
    rng = np.random.default_rng(21)
    z = rng.uniform(0.0, 10.0, (P.shape[0], 37))
    z[:, 0], z[:, 1] = 1e-3, 1100.0
    return P, z.reshape(-1), np.arange(P.shape[0] + 1, dtype=np.int64) * 37


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_components_forward_vs_quadrature(lib, prec):
    P, z, offs = _rows()
    zin = z if prec == "fp64" else z.astype(np.float32)
    ref = oracle.quad_distances(P, zin.astype(np.float64), offs)
    res = lib.distances(_t(P), _t(zin), _t(offs), outputs=ALL, precision=prec)
    torch.cuda.synchronize()
    assert int(res["status"].abs().sum()) == 0
    _check(res, ref, TOL64 if prec == "fp64" else TOL32, prec, (P, offs))


def test_components_loglike_and_refusals(lib):
    P, z, offs = _rows()
    z32 = np.maximum(z, 1e-3).astype(np.float32)
    mu = oracle.quad_distances(P, z32.astype(np.float64), offs)[:, 5]
    m = (mu - 19.3 + np.random.default_rng(4).normal(0.0, 0.1, z.size)).astype(np.float32)
    res = lib.gauss_loglike(_t(P), _t(z32), _t(m), _t(offs), M=-19.3, sigma=0.1, grad=False, want_mu=True,
                            precision="fp32")
    torch.cuda.synchronize()
    rows = np.repeat(np.arange(P.shape[0]), 37)
    want = np.array([np.sum(-0.5 * ((m[rows == b] - mu[rows == b] + 19.3) / 0.1) ** 2
                            - np.log(0.1 * np.sqrt(2 * np.pi))) for b in range(P.shape[0])])
    got = res["loglike"].cpu().numpy()
    # mu within 1e-5 mag per pair: the sum of the squared residuals moves by at most 2 |r| 1e-5 / sigma^2 each
    bound = np.array([np.sum(2 * np.abs(m[rows == b] - mu[rows == b] + 19.3) * 1e-5 / 0.01 + 1e-6)
                      for b in range(P.shape[0])])
    assert np.all(np.abs(got - want) <= bound), np.abs(got - want) / bound
    with pytest.raises(RuntimeError):
        lib.distances_vjp(_t(P), _t(z32), {"mu": _t(np.ones_like(z32))}, _t(offs))
    with pytest.raises(RuntimeError):
        lib.gauss_loglike(_t(P), _t(z32), _t(m), _t(offs), grad=True)
