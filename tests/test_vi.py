"""The variational-inference step (Sec. 4 model, flat prior, Gaussian guide)
captured in a CUDA graph: it runs through the fused log-likelihood kernel,
raises the ELBO and moves the guide towards the parameters that generated the
mock magnitudes.  The magnitudes come from the Carlson oracle at the truth."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


def _data(N=20000, seed=5, truth=(70.0, 0.3, 0.7, 5e-5), M=-19.3, sigma=0.1):
    rng = np.random.default_rng(seed)
    z = rng.uniform(0.01, 1.5, N)
    mu = oracle.carlson_distances(np.array([truth]), z, np.array([0, N]))[:, 5]
    return z, mu + M + rng.normal(0.0, sigma, N)


def test_vi_graph_step_converges(lib):
    from paper_2212_01937_gb300 import vi
    truth = (70.0, 0.3, 0.7, 5e-5)
    z, m_obs = _data(truth=truth)
    dev = torch.device("cuda:0")
    torch.manual_seed(0)
    centre, scale = vi.default_guide(truth)
    opt = vi.GaussianVI(torch.tensor(z, dtype=torch.float32, device=dev),
                        torch.tensor(m_obs, device=dev), centre, scale, samples=64, lr=0.05, graph=True)
    n0 = lib.launch_count()
    opt.step()
    torch.cuda.synchronize()
    elbo0 = float(opt.elbo)
    assert float(opt.valid) == 64
    for _ in range(400):
        opt.step()
    torch.cuda.synchronize()
    # graph replays do not pass through the host entry points
    assert lib.launch_count() == n0
    mean, std = opt.posterior()
    mean = mean.cpu().numpy()
    assert float(opt.elbo) > elbo0
    assert abs(mean[0] - truth[0]) < 0.5, mean
    assert abs(mean[1] - truth[1]) < 0.1, mean
    assert abs(mean[2] - truth[2]) < 0.15, mean
