"""The Sec. 4 model with latent redshifts: the per-pair derivative of the
magnitude log-likelihood with respect to the redshift (lcdm_gauss_loglike_dz,
through the C ABI) against the oracle; the ELBO gradient of the
partial-MVN guide against finite differences; and a VI run on mock data.

Tolerances: d loglike / dz per pair within (1e-9 FP64, 2e-5 FP32) relative
in d mu/dz plus an absolute error of (1e-11, 2e-5 x condition number) mag
on the residual, against the oracle's d mu/dz (the integrand of eq. 2.3
through the curvature map) and mu.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_01937_gb300 import workloads

from test_gpu_parity import _t, mu_cond

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_loglike_grad_z_vs_oracle(lib, prec):
    b = workloads.general_batch(B=5, n=64, seed=13, zmax=3.0)
    rng = np.random.default_rng(5)
    dt = np.float64 if prec == "fp64" else np.float32
    z = np.maximum(b.z, 1e-3).astype(dt)        # the likelihood needs z > 0 (mu = -inf at z = 0)
    z[::17] = np.resize([1e-4, 2e-3, 0.05, 1.0], z[::17].size)
    zq = z.astype(np.float64)
    ref = oracle.quad_distances(b.params, zq, b.offsets)
    mu = ref[:, 5]
    m = mu - 19.3 + rng.normal(0.0, 0.1, z.size)
    m = m.astype(dt)
    sigma, M = 0.1, -19.3
    res = lib.gauss_loglike(_t(b.params), _t(z), _t(m), None, M=M, sigma=sigma, grad=True, grad_z=True,
                            want_mu=True, layout="dense", precision=prec)
    plain = lib.gauss_loglike(_t(b.params), _t(z), _t(m), None, M=M, sigma=sigma, grad=True, layout="dense",
                              precision=prec)
    torch.cuda.synchronize()
    assert int(res["status"].abs().sum()) == 0
    # the log-likelihood and its parameter gradient are those of lcdm_gauss_loglike
    assert torch.equal(res["loglike"], plain["loglike"]) and torch.equal(res["grad"], plain["grad"])
    gz = res["grad_z"].double().cpu().numpy()
    dmu = oracle.dmu_dz(b.params, zq, b.offsets)
    r = m.astype(np.float64) - mu - M
    want = r / sigma ** 2 * dmu
    rel_d, abs_r = (1e-9, 1e-11) if prec == "fp64" else (2e-5, 2e-5)
    cond = mu_cond(ref, b.params, b.offsets)
    bound = (rel_d * np.abs(r) + abs_r * cond) * np.abs(dmu) / sigma ** 2
    assert np.all(np.abs(gz - want) <= bound), (prec, np.max(np.abs(gz - want) / bound))


def _mock(N, seed, exact=True):
    truth = (0.3, 0.7)
    mu = None
    if exact:
        p = np.array([[70.0, truth[0], truth[1], 0.0]])
        mu = lambda z: oracle.carlson_distances(p, z)[:, 5]
    return workloads.bhm_supernovae(N=N, seed=seed, truth=truth, mu=mu)


def test_bhm_elbo_gradient_vs_finite_differences(lib):
    """With the noise held fixed the ELBO estimate is a deterministic function
    of the guide parameters: its reparameterisation gradient (FP64 path)
    against central differences of the same estimate."""
    from paper_2212_01937_gb300 import bhm
    d = _mock(48, seed=3)
    dev = "cuda:0"
    vi = bhm.PMVNGuideVI(torch.tensor(d.extra["z_hat"], device=dev), torch.tensor(d.m_obs, device=dev),
                         samples=3, precision="fp64", graph=False)
    torch.manual_seed(0)
    vi._draw()
    # move away from the initial point so that b and the off-diagonal of L matter
    g = torch.Generator(device="cpu").manual_seed(1)
    vi.b.copy_(0.3 * torch.randn(vi.N, 2, generator=g, dtype=torch.float64).to(dev))
    vi.l[1] = 0.02
    grads = {k: v.clone() for k, v in vi.gradients().items()}

    def elbo():
        vi.gradients()
        return float(vi.elbo)

    checks = [("m", (0,)), ("m", (1,)), ("l", (0,)), ("l", (1,)), ("l", (2,)), ("a", (5,)), ("a", (31,)),
              ("b", (7, 0)), ("b", (20, 1)), ("c", (11,)), ("c", (40,))]
    for name, idx in checks:
        v = getattr(vi, name)
        x0 = float(v[idx])
        h = 1e-6 * max(1.0, abs(x0))
        v[idx] = x0 + h
        fp = elbo()
        v[idx] = x0 - h
        fm = elbo()
        v[idx] = x0
        fd = (fp - fm) / (2 * h)
        got = float(grads[name][idx])
        assert abs(got - fd) <= 1e-5 * max(abs(fd), 1.0), (name, idx, got, fd)


def test_bhm_vi_recovers_cosmology(lib):
    from paper_2212_01937_gb300 import bhm
    d = _mock(4000, seed=11)
    dev = "cuda:0"
    torch.manual_seed(2)
    vi = bhm.PMVNGuideVI(torch.tensor(d.extra["z_hat"], device=dev), torch.tensor(d.m_obs, device=dev),
                         samples=4, lr=0.01)
    for _ in range(3000):
        vi.step()
    torch.cuda.synchronize()
    mean, cov = vi.posterior()
    mean, std = mean.cpu().numpy(), np.sqrt(np.diag(cov.cpu().numpy()))
    truth = np.array(d.extra["truth"])
    assert np.all(std > 1e-3) and np.all(std < 0.3), std
    assert np.all(np.abs(mean - truth) <= 4 * std + 0.02), (mean, std)
    # the latent redshifts move towards the truth from the photometric estimates
    zg = vi.redshifts().double().cpu().numpy()
    zt, zh = d.z, d.extra["z_hat"]
    assert np.sqrt(np.mean((zg - zt) ** 2)) < np.sqrt(np.mean((zh - zt) ** 2))


OUTS = ("d_C", "t", "X", "d_M", "d_L", "mu")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_distances_grad_z_vs_oracle(lib, prec):
    """lcdm_distances_vjp_dz: sum_o cot_o d out_o/dz per pair against the
    oracle's integrands (eqs. 2.3-2.5 at the upper limit) through the
    curvature map; z = 0 included (d mu/dz counts as 0 there).  The parameter
    gradient is that of lcdm_distances_vjp."""
    b = workloads.general_batch(B=5, n=64, seed=17, zmax=5.0)
    dt = np.float64 if prec == "fp64" else np.float32
    z = b.z.astype(dt)
    z[::23] = 0.0
    z[5::29] = 1100.0
    zq = z.astype(np.float64)
    rng = np.random.default_rng(7)
    cot = {n: rng.normal(size=z.size).astype(dt) for n in OUTS}
    d = oracle.dout_dz(b.params, zq, b.offsets)
    want = sum(cot[n].astype(np.float64) * d[:, k] for k, n in enumerate(OUTS))
    res = lib.distances_vjp(_t(b.params), _t(z), {n: _t(v) for n, v in cot.items()}, _t(b.offsets),
                            grad_z=True, precision=prec)
    plain = lib.distances_vjp(_t(b.params), _t(z), {n: _t(v) for n, v in cot.items()}, _t(b.offsets),
                              precision=prec)
    torch.cuda.synchronize()
    assert int(res["status"].abs().sum()) == 0
    assert torch.equal(res["grad"], plain["grad"])
    ref = oracle.quad_distances(b.params, zq, b.offsets)
    cond = mu_cond(ref, b.params, b.offsets)
    rel = 1e-10 if prec == "fp64" else 2e-5
    bound = rel * cond * sum(np.abs(cot[n].astype(np.float64) * d[:, k]) for k, n in enumerate(OUTS))
    got = res["grad_z"].double().cpu().numpy()
    assert np.all(np.abs(got - want) <= bound + 1e-300), (prec, np.max(np.abs(got - want) / bound))


def test_autograd_redshift_gradient(lib):
    """torch.autograd through lcdm.Distances with redshifts that require a
    gradient (FP64): z.grad against the oracle's z-derivatives."""
    b = workloads.general_batch(B=4, n=50, seed=19)
    params = _t(b.params).requires_grad_(True)
    z = _t(b.z).requires_grad_(True)
    off = _t(b.offsets)
    rng = np.random.default_rng(9)
    w = {n: rng.normal(size=b.nnz) for n in ("d_C", "t", "mu")}
    d_C, t, mu = lib.distances_autograd(params, z, off, outputs=("d_C", "t", "mu"), precision="fp64")
    loss = sum((_t(w[n]) * v).sum() for n, v in zip(("d_C", "t", "mu"), (d_C, t, mu)))
    loss.backward()
    torch.cuda.synchronize()
    d = oracle.dout_dz(b.params, b.z, b.offsets)
    want = w["d_C"] * d[:, 0] + w["t"] * d[:, 1] + w["mu"] * d[:, 5]
    scale = np.abs(w["d_C"] * d[:, 0]) + np.abs(w["t"] * d[:, 1]) + np.abs(w["mu"] * d[:, 5])
    got = z.grad.cpu().numpy()
    assert np.all(np.abs(got - want) <= 1e-10 * scale), np.max(np.abs(got - want) / scale)
    assert params.grad is not None and torch.isfinite(params.grad).all()
