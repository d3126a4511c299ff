"""Variational inference over (H0, Omega_m0, Omega_L0, Omega_r0) from mock
supernova magnitudes (Sec. 4), one step per CUDA-graph replay.

The guide is a mean-field Gaussian over theta = centre + scale * u, with
u ~ N(m, diag(exp(2 s))): the fixed affine map only puts the four parameters
on comparable numerical scales for the optimiser.  One step:

  1. eps ~ N(0, 1) [S, 4] (torch's CUDA generator, graph-safe);
     theta_s = centre + scale * (m + exp(s) eps_s);
  2. lcdm_gauss_loglike over the shared redshift set: loglike_s and
     d loglike_s / d theta_s for all S samples in one launch (fused forward +
     adjoint, FP64 per-sample reductions);
  3. ELBO = mean_s loglike_s + sum(s) (Gaussian entropy up to a constant,
     flat prior), with the reparameterisation gradients
       dELBO/dm = mean_s g_s * scale,  dELBO/ds = mean_s g_s * scale * exp(s) eps_s + 1;
     samples without a valid cosmology (status != 0) get weight 0;
  4. Adam ascent on (m, s).

Every buffer is allocated once, so the whole step is captured in one CUDA
graph (graph=True) and replayed; graph=False runs the same step eagerly.
"""
import math

import torch

from . import lcdm, shard

PARAM_NAMES = ("H0", "Om", "OL", "Or")


class GaussianVI:
    def __init__(self, z, m_obs, centre, scale, M=-19.3, sigma=0.1, samples=256, lr=0.05,
                 init_log_std=-1.0, precision="fp32", graph=True, betas=(0.9, 0.999), eps=1e-8, group=None):
        dev = z.device
        if not z.is_cuda:
            raise ValueError("z must be a CUDA tensor")
        f64 = dict(dtype=torch.float64, device=dev)
        self.S = int(samples)
        self.M, self.sigma = float(M), float(sigma)
        self.centre = torch.as_tensor(centre, **f64).reshape(4)
        self.scale = torch.as_tensor(scale, **f64).reshape(4)
        self.m = torch.zeros(4, **f64)
        self.s = torch.full((4,), float(init_log_std), **f64)
        self.lr, self.b1, self.b2, self.adam_eps = float(lr), betas[0], betas[1], float(eps)
        self.t = torch.zeros((), **f64)
        self.mom = torch.zeros(8, **f64)
        self.vel = torch.zeros(8, **f64)
        self.noise = torch.zeros(self.S, 4, **f64)
        self.params = torch.zeros(self.S, 4, **f64)
        self.elbo = torch.zeros((), **f64)
        self.valid = torch.zeros((), **f64)
        self.call = lcdm.Call(self.params, z, layout="shared", precision=precision)
        self.m_obs = m_obs.to(device=dev, dtype=self.call.dtype).contiguous()
        # with a process group, z and m_obs are this rank's share of the
        # supernovae; the per-sample sums are added over the ranks by one
        # all-reduce (shard.allreduce_loglike), and every rank must seed its
        # CUDA generator alike so that all draw the same guide samples
        self.group = group
        self.graph = None
        if graph:
            self._capture()

    # ------------------------------------------------------------------
    def _body(self):
        torch.randn(self.S, 4, out=self.noise)
        std = torch.exp(self.s)
        u = self.m + std * self.noise
        self.params.copy_(self.centre + self.scale * u)
        res = lcdm.gauss_loglike(self.params, None, self.m_obs, M=self.M, sigma=self.sigma, grad=True,
                                 call=self.call)
        ll, g = res["loglike"], res["grad"]
        if self.group is not None:
            shard.allreduce_loglike(ll, g, self.group)
        ok = (self.call.status == 0) & torch.isfinite(ll) & torch.isfinite(g).all(dim=1)
        w = ok.to(torch.float64)
        n = w.sum().clamp(min=1.0)
        w = w / n
        ll0 = torch.where(ok, ll, torch.zeros_like(ll))
        g0 = torch.where(ok[:, None], g, torch.zeros_like(g)) * self.scale
        self.elbo.copy_((w * ll0).sum() + self.s.sum())
        self.valid.copy_(n)
        gm = (w[:, None] * g0).sum(dim=0)
        gs = (w[:, None] * g0 * std * self.noise).sum(dim=0) + 1.0
        grad = torch.cat([gm, gs])
        # Adam, ascending the ELBO
        self.t.add_(1.0)
        self.mom.mul_(self.b1).add_((1.0 - self.b1) * grad)
        self.vel.mul_(self.b2).add_((1.0 - self.b2) * grad * grad)
        mhat = self.mom / (1.0 - torch.pow(self.b1, self.t))
        vhat = self.vel / (1.0 - torch.pow(self.b2, self.t))
        step = self.lr * mhat / (torch.sqrt(vhat) + self.adam_eps)
        self.m.add_(step[:4])
        self.s.add_(step[4:])

    def _capture(self):
        side = torch.cuda.Stream(device=self.params.device)
        side.wait_stream(torch.cuda.current_stream(self.params.device))
        state = [x.clone() for x in (self.m, self.s, self.t, self.mom, self.vel)]
        with torch.cuda.stream(side):
            for _ in range(2):       # warm-up outside the capture (lazy init, autotune cache)
                self._body()
        torch.cuda.current_stream(self.params.device).wait_stream(side)
        for x, v in zip((self.m, self.s, self.t, self.mom, self.vel), state):
            x.copy_(v)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._body()

    # ------------------------------------------------------------------
    def step(self):
        """One VI step (graph replay when captured)."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self._body()

    def posterior(self):
        """Guide mean and standard deviation in parameter units [4] each."""
        mean = self.centre + self.scale * self.m
        std = self.scale * torch.exp(self.s)
        return mean, std

    @property
    def pairs_per_step(self):
        return self.S * self.call.n


def default_guide(truth=(70.0, 0.3, 0.7, 5e-5)):
    """Centre at a perturbed guess and per-parameter scales for the affine map."""
    centre = (truth[0] * 1.02, truth[1] * 1.1, truth[2] * 0.95, truth[3] * 1.2)
    scale = (1.0, 0.01, 0.01, 1e-5)
    return centre, scale
