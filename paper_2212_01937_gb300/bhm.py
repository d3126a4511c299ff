"""Variational inference for the supernova model of Sec. 4 with latent
redshifts, one step per CUDA-graph replay.

Model (Sec. 4): for each supernova n, a latent redshift z_n with a gamma
prior (shape alpha, rate beta), an observed redshift zhat_n ~ N(z_n,
(1+z_n)^2 sigma_z^2) and an observed distance modulus muhat_n ~
N(mu(z_n; Om, OL), sigma_mu^2); radiationless LCDM with the closure, H0 fixed
(it is degenerate with the absolute magnitude), a flat prior on (Om, OL) over
universes with a Big Bang.

Guide: a partial multivariate normal.  theta = (Om, OL) ~ N(m, L L^T); for
each supernova the log-redshift w_n = log z_n given theta is
N(a_n + b_n . (theta - m), exp(2 c_n)): the correlations of the two global
parameters with every latent redshift are kept, those between supernovae
are not.  One step, for S guide samples:

  1. eps ~ N(0, 1) [S, 2] and [S, N]; delta = L eps_theta; theta = m + delta;
     w = a + b delta + exp(c) eps_w; z = exp(w);
  2. lcdm_gauss_loglike_dz over the [S, N] dense batch (one row per sample):
     the distance-modulus log-likelihood, its gradient w.r.t. (Om, OL) and
     its derivative w.r.t. each latent redshift (d mu/dz from the integrand
     of eq. 2.3); the redshift likelihood, the gamma prior and the Jacobian
     of z = exp(w) are elementwise terms;
  3. reparameterisation gradients of ELBO = E[log p(data, theta, z) + sum w]
     + log det L + sum c (+ const); samples without a valid cosmology get
     weight 0;
  4. Adam ascent on (m, log-Cholesky of L, a, b, c).

Every buffer is allocated once, so the step is captured in one CUDA graph.
"""
import math

import torch

from . import lcdm


class PMVNGuideVI:
    def __init__(self, z_hat, mu_hat, H0=70.0, alpha=2.0, beta=3.0, sigma_mu=0.14, sigma_z=0.04, samples=4,
                 lr=0.01, init=(0.35, 0.6), init_std=0.05, precision="fp32", graph=True, betas=(0.9, 0.999),
                 eps=1e-8):
        dev = z_hat.device
        if not z_hat.is_cuda:
            raise ValueError("z_hat must be a CUDA tensor")
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        f64 = dict(dtype=torch.float64, device=dev)
        fT = dict(dtype=self.dtype, device=dev)
        self.S, self.N = int(samples), int(z_hat.numel())
        self.H0, self.alpha, self.beta = float(H0), float(alpha), float(beta)
        self.smu, self.sz = float(sigma_mu), float(sigma_z)
        self.zhat = z_hat.to(**fT).reshape(-1).contiguous()
        # distance moduli, one copy per sample row (the dense layout indexes them like z)
        self.muhat = mu_hat.to(**fT).reshape(1, -1).repeat(self.S, 1).reshape(-1).contiguous()
        # variational parameters
        self.m = torch.tensor(init, **f64)
        self.l = torch.tensor([math.log(init_std), 0.0, math.log(init_std)], **f64)   # L00, L10, L11 (log-diag)
        zh = self.zhat.double().clamp(min=1e-3)
        self.a = torch.log(zh).to(**fT)
        self.b = torch.zeros(self.N, 2, **fT)
        self.c = torch.log((self.sz * (1.0 + zh) / zh).clamp(max=1.0)).to(**fT)
        self.lr, self.b1, self.b2, self.adam_eps = float(lr), betas[0], betas[1], float(eps)
        self.t = torch.zeros((), **f64)
        self.state = {k: (torch.zeros_like(v), torch.zeros_like(v)) for k, v in self._vars().items()}
        # per-step buffers
        self.eps_t = torch.zeros(self.S, 2, **f64)
        self.eps_w = torch.zeros(self.S, self.N, **fT)
        self.params = torch.zeros(self.S, 4, **f64)
        self.z = torch.zeros(self.S * self.N, **fT)
        self.elbo = torch.zeros((), **f64)
        self.valid = torch.zeros((), **f64)
        self.call = lcdm.Call(self.params, self.z, layout="dense", precision=precision)
        self.ws = lcdm.loglike_dz_workspace(self.call)
        self.graph = None
        if graph:
            self._capture()

    def _vars(self):
        return {"m": self.m, "l": self.l, "a": self.a, "b": self.b, "c": self.c}

    def L(self):
        l = self.l
        return torch.stack([torch.stack([torch.exp(l[0]), torch.zeros_like(l[0])]),
                            torch.stack([l[1], torch.exp(l[2])])])

    # ------------------------------------------------------------------
    def _body(self):
        self._draw()
        self._adam(self.gradients())

    def _draw(self):
        torch.randn(self.S, 2, out=self.eps_t)
        torch.randn(self.S, self.N, out=self.eps_w)

    def gradients(self):
        """ELBO estimate (into self.elbo) and its gradients w.r.t. the guide
        parameters for the current noise draw."""
        S, N = self.S, self.N
        L = self.L()
        delta = self.eps_t @ L.T                                    # [S, 2]
        theta = self.m + delta
        dT = delta.to(self.dtype)
        sc = torch.exp(self.c)
        w = self.a + dT @ self.b.T + sc * self.eps_w                # [S, N]
        z = torch.exp(w)
        self.z.copy_(z.reshape(-1))
        self.params[:, 0] = self.H0
        self.params[:, 1:3] = theta
        self.params[:, 3] = 0.0
        res = lcdm.gauss_loglike(self.params, None, self.muhat, M=0.0, sigma=self.smu, grad=True, grad_z=True,
                                 call=self.call, workspace=self.ws)
        ll, g, gz = res["loglike"], res["grad"], res["grad_z"].reshape(S, N)
        # redshift likelihood N(zhat; z, (1+z)^2 sz^2), gamma prior, Jacobian of z = exp(w)
        x = 1.0 + z
        r = (self.zhat - z) / (x * self.sz)
        lz = -0.5 * r * r - torch.log(x) + (self.alpha - 1.0) * w - self.beta * z + w
        dz = gz + r / (x * self.sz) + r * r / x - 1.0 / x + (self.alpha - 1.0) / z - self.beta
        gw = dz * z + 1.0                                           # d/dw, the Jacobian term included
        ok = (self.call.status == 0) & torch.isfinite(ll) & torch.isfinite(g[:, 1:3]).all(dim=1) \
            & torch.isfinite(gw).all(dim=1)
        wgt = ok.to(torch.float64)
        n = wgt.sum().clamp(min=1.0)
        wgt = wgt / n
        logp = torch.where(ok, ll + lz.sum(dim=1, dtype=torch.float64), torch.zeros_like(ll))
        ent = self.l[0] + self.l[2] + self.c.sum(dtype=torch.float64)
        self.elbo.copy_((wgt * logp).sum() + ent)
        self.valid.copy_(n)
        gth = torch.where(ok[:, None], g[:, 1:3], torch.zeros_like(g[:, 1:3]))
        gw = torch.where(ok[:, None], gw, torch.zeros_like(gw))
        wT = wgt.to(self.dtype)
        # reparameterisation gradients
        gdelta = gth + (gw @ self.b).double()                       # d logp / d delta [S, 2]
        gm = (wgt[:, None] * gth).sum(dim=0)
        gL = (wgt[:, None, None] * gdelta[:, :, None] * self.eps_t[:, None, :]).sum(dim=0)
        gl = torch.stack([gL[0, 0] * torch.exp(self.l[0]) + 1.0, gL[1, 0], gL[1, 1] * torch.exp(self.l[2]) + 1.0])
        gwW = gw * wT[:, None]
        ga = gwW.sum(dim=0)
        gb = gwW.T @ dT
        gc = (gwW * self.eps_w).sum(dim=0) * sc + 1.0
        return {"m": gm, "l": gl, "a": ga, "b": gb, "c": gc}

    def _adam(self, grads):
        self.t.add_(1.0)
        c1 = 1.0 - torch.pow(self.b1, self.t)
        c2 = 1.0 - torch.pow(self.b2, self.t)
        for k, v in self._vars().items():
            g = grads[k].to(v.dtype)
            mo, ve = self.state[k]
            mo.mul_(self.b1).add_((1.0 - self.b1) * g)
            ve.mul_(self.b2).add_((1.0 - self.b2) * g * g)
            step = self.lr * (mo / c1.to(v.dtype)) / (torch.sqrt(ve / c2.to(v.dtype)) + self.adam_eps)
            v.add_(step)

    def _capture(self):
        dev = self.m.device
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        saved = {k: v.clone() for k, v in self._vars().items()}
        saved_state = {k: (a.clone(), b.clone()) for k, (a, b) in self.state.items()}
        t0 = self.t.clone()
        with torch.cuda.stream(side):
            for _ in range(2):       # warm-up outside the capture
                self._body()
        torch.cuda.current_stream(dev).wait_stream(side)
        for k, v in self._vars().items():
            v.copy_(saved[k])
            self.state[k][0].copy_(saved_state[k][0])
            self.state[k][1].copy_(saved_state[k][1])
        self.t.copy_(t0)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._body()

    # ------------------------------------------------------------------
    def step(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self._body()

    def posterior(self):
        """Guide mean and covariance of (Om, OL)."""
        L = self.L()
        return self.m.clone(), L @ L.T

    def redshifts(self):
        """Guide median of each latent redshift (at theta = m)."""
        return torch.exp(self.a)

    @property
    def pairs_per_step(self):
        return self.S * self.N
