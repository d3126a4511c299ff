"""Seven-column rows (the further components of fn4, w = -1/3 and -2/3):
forward distances, the magnitude log-likelihood, and the derivatives with
respect to all six densities (Om, OL, Or, Ok, Os, Ox, each independent)
through the C ABI against the oracle (its Leibniz-rule gradients
differentiate Os and Ox as well).  Tolerances as for the five-column path
(test_gpu_parity.py)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_01937_gb300 import workloads

from test_gpu_parity import COLS, TOL32, TOL64, _check, _t, jac_tol

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
    # the gradient of the log-likelihood: r/sigma^2 d mu / d theta summed per row
    _, J = oracle.quad_distances(P, z32.astype(np.float64), offs, grad=True)
    r = (m.astype(np.float64) - mu + 19.3) / 0.1
    gw = np.array([((r[rows == b] / 0.1)[:, None] * J[rows == b, 5, :]).sum(axis=0) for b in range(P.shape[0])])
    res = lib.gauss_loglike(_t(P), _t(z32), _t(m), _t(offs), M=-19.3, sigma=0.1, grad=True, precision="fp32")
    torch.cuda.synchronize()
    gg = res["grad"].cpu().numpy()
    # bound per entry: each pair's residual moves with its mu (<= 1e-5 mag) and
    # its d mu / d theta with the Jacobian bound (3e-5 + 2e-6/z of the row max)
    zq = z32.astype(np.float64)
    jrow = np.abs(J[:, 5, :]).max(axis=1, keepdims=True)
    per = np.abs(J[:, 5, :]) * 1e-5 / 0.01 + np.abs(r / 0.1)[:, None] * jrow * (3e-5 + 2e-6 / zq)[:, None]
    gb = np.array([per[rows == b].sum(axis=0) for b in range(P.shape[0])])
    for b in range(P.shape[0]):
        c = np.ones(P.shape[1], dtype=bool)
        if P[b, 3] == 0:
            c[3] = False                      # a radiationless row has no Omega_r0 direction
            assert np.isnan(gg[b, 3])
        assert np.all(np.abs(gg[b, c] - gw[b, c]) <= gb[b, c]), (b, np.abs(gg[b] - gw[b]) / gb[b])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_components_jacobian_vs_leibniz_oracle(lib, prec):
    """Per-pair Jacobians with respect to (H0, Om, OL, Or, Ok, Os, Ox)."""
    P, z, offs = _rows()
    zin = z if prec == "fp64" else z.astype(np.float32)
    zq = zin.astype(np.float64)
    _, J = oracle.quad_distances(P, zq, offs, grad=True)
    res = lib.distances_jac(_t(P), _t(zin), _t(offs), outputs=("d_C", "t", "X", "mu"), precision=prec)
    torch.cuda.synchronize()
    assert int(res["status"].abs().sum()) == 0
    rows = np.repeat(np.arange(P.shape[0]), np.diff(offs))
    rad = P[rows, 3] > 0
    for n in (("d_C", "t", "X", "mu") if prec == "fp64" else ("d_C", "t", "mu")):
        got = res["jac"][n].double().cpu().numpy()
        want = J[:, COLS[n], :]
        assert np.all(np.isnan(got[~rad, 3]))
        got[~rad, 3] = want[~rad, 3] = 0.0
        err = np.abs(got - want).max(axis=1) / np.abs(want).max(axis=1)
        assert np.all(err <= jac_tol(prec, zq, n)), (prec, n, err.max())
