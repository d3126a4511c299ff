"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds none of the distance method's arithmetic: it draws
cosmologies and redshifts, rejects draws without a Big Bang by checking the
sign of Q(a) = a^4 E^2 on (0, 1] (no roots of E^2, no Carlson integrals), and
makes mock supernova magnitudes from a low-redshift cosmographic series (not
from the method).  Both the CUDA path's tests/benchmarks and the oracle's
tests take their inputs from here.

Every generator draws, per cosmology and in this order: Omega_m0, Omega_L0,
log10 Omega_r0, H0; then the redshifts.  Rejected cosmologies are redrawn.

Parameter rows are (H0 [km/s/Mpc], Omega_m0, Omega_L0, Omega_r0) with
Omega_k0 = 1 - Omega_m0 - Omega_L0 - Omega_r0 (closure, Sec. 2.1), or with a
fifth column Omega_k0 when given explicitly.
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

C_KMS = 299792.458


def q_min(Om, OL, Or, Ok):
    """min over a in (0, 1] of Q(a) = Or + Om a + Ok a^2 + OL a^4.

    A universe has a Big Bang connected smoothly to z = 0 (Sec. 3, Fig. 1)
    iff Q > 0 on (0, 1] (for Or = 0 the end point a -> 0 is excluded and Q/a
    is checked there instead).  Stationary points solve
    Q'(a) = Om + 2 Ok a + 4 OL a^3 = 0."""
    cands = [1.0]
    crit = np.roots([4.0 * OL, 0.0, 2.0 * Ok, Om]) if OL != 0 else (
        np.array([-Om / (2.0 * Ok)]) if Ok != 0 else np.array([]))
    for c in np.atleast_1d(crit):
        if abs(c.imag) < 1e-12 and 0.0 < c.real < 1.0:
            cands.append(c.real)
    vals = [Or + Om * a + Ok * a * a + OL * a ** 4 for a in cands]
    if Or == 0.0:
        vals.append(Om)  # limit of Q(a)/a at a -> 0
    else:
        vals.append(Or)
    return min(vals)


def has_big_bang(Om, OL, Or, Ok=None):
    if Ok is None:
        Ok = 1.0 - Om - OL - Or
    return q_min(Om, OL, Or, Ok) > 0.0


def ol_critical(Om, Or, lo=0.0, hi=10.0, iters=200):
    """Largest Omega_L0 (closure) that still has a Big Bang, by bisection on
    the sign of min Q (the no-Big-Bang boundary of Fig. 1)."""
    assert has_big_bang(Om, lo, Or)
    while has_big_bang(Om, hi, Or):
        hi *= 2.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if has_big_bang(Om, mid, Or):
            lo = mid
        else:
            hi = mid
        if hi - lo <= 1e-15 * hi:
            break
    return lo


def mock_mu(z, H0, Om, OL, Or):
    """Distance modulus from the second-order cosmographic series
    d_L ~ (c z / H0) (1 + (1 - q0) z / 2), q0 = Om/2 + Or - OL.  Used only to
    make mock magnitudes (the stand-in for the paper's mock SN sets); it is
    not the method under test."""
    q0 = 0.5 * Om + Or - OL
    dl = C_KMS * z / H0 * (1.0 + 0.5 * (1.0 - q0) * z)
    return 5.0 * np.log10(dl) + 25.0


@dataclass
class Batch:
    """A ragged (CSR) batch of (cosmology, redshift) pairs."""
    name: str
    params: np.ndarray                 # [B, 4 or 5] float64
    z: np.ndarray                      # [nnz] float64
    offsets: np.ndarray                # [B+1] int64
    m_obs: Optional[np.ndarray] = None  # [nnz] mock magnitudes (loglike workloads)
    M: float = -19.3
    sigma: float = 0.1
    extra: dict = field(default_factory=dict)

    @property
    def B(self):
        return self.params.shape[0]

    @property
    def nnz(self):
        return self.z.size


def _draw_cosmo(rng, Om_rng=(0.05, 0.6), OL_rng=(0.0, 1.2), lOr_rng=(-5.0, -4.0),
                H0_rng=(60.0, 80.0)):
    while True:
        Om = rng.uniform(*Om_rng)
        OL = rng.uniform(*OL_rng)
        Or = 10.0 ** rng.uniform(*lOr_rng)
        H0 = rng.uniform(*H0_rng)
        if has_big_bang(Om, OL, Or):
            return H0, Om, OL, Or


def flat_radiationless(n=10_000, seed=0):
    """One flat radiationless cosmology (70, 0.3, 0.7, 0); z ~ U(0.01, 2)."""
    rng = np.random.default_rng(seed)
    params = np.array([[70.0, 0.3, 0.7, 0.0]])
    z = rng.uniform(0.01, 2.0, n)
    return Batch("flat-radiationless-1x%d" % n, params, z, np.array([0, n], dtype=np.int64))


def general_batch(B=4096, n=1024, seed=2, zmax=10.0):
    """General LCDM+radiation+curvature batch: Om ~ U(.05,.6), OL ~ U(0,1.2),
    Or ~ logU(1e-5,1e-4), H0 ~ U(60,80), n redshifts each z ~ U(0, zmax)."""
    rng = np.random.default_rng(seed)
    params = np.zeros((B, 4))
    z = np.zeros((B, n))
    for b in range(B):
        H0, Om, OL, Or = _draw_cosmo(rng)
        params[b] = (H0, Om, OL, Or)
        z[b] = rng.uniform(0.0, zmax, n)
    return Batch("lcdm-rad-curv-%dx%d" % (B, n), params, z.reshape(-1),
                 np.arange(B + 1, dtype=np.int64) * n)


def supernovae(N=1_000_000, seed=1, truth=(70.0, 0.3, 0.7, 5e-5), M=-19.3, sigma=0.1):
    """N mock SNe Ia: z ~ U(0.01, 1.5), m_obs = mu_mock(z; truth) + M + N(0, sigma^2).
    The stand-in for the Sec. 4 mock sets (up to 10^6 SNe)."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(0.01, 1.5, N)
    H0, Om, OL, Or = truth
    m_obs = mock_mu(z, H0, Om, OL, Or) + M + rng.normal(0.0, sigma, N)
    return Batch("sn-ia-%d" % N, np.array([truth]), z, np.array([0, N], dtype=np.int64),
                 m_obs=m_obs, M=M, sigma=sigma, extra={"truth": truth})


def ragged_batch(B=16384, seed=3, nmax_exp=5.0, M=-19.3, sigma=0.1):
    """Ragged batch: cosmologies as general_batch; row length floor(10^U(0, nmax_exp));
    z ~ U(0, 3); per-row mock magnitudes from the row's own cosmology."""
    rng = np.random.default_rng(seed)
    params = np.zeros((B, 4))
    lens = np.zeros(B, dtype=np.int64)
    zs, ms = [], []
    for b in range(B):
        H0, Om, OL, Or = _draw_cosmo(rng)
        params[b] = (H0, Om, OL, Or)
        n = int(np.floor(10.0 ** rng.uniform(0.0, nmax_exp)))
        lens[b] = n
        zb = rng.uniform(0.0, 3.0, n)
        zs.append(zb)
        zb_safe = np.maximum(zb, 1e-8)
        ms.append(mock_mu(zb_safe, H0, Om, OL, Or) + M + rng.normal(0.0, sigma, n))
    offsets = np.zeros(B + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lens)
    return Batch("ragged-%d" % B, params, np.concatenate(zs), offsets,
                 m_obs=np.concatenate(ms), M=M, sigma=sigma)


def precision_stress(B=10_000, n=10_000, seed=4):
    """Precision stress: half the cosmologies within 1e-6 of flatness
    (Ok ~ U(-1e-6, 1e-6), OL = 1 - Om - Or - Ok), half just inside the
    no-Big-Bang boundary (OL = OL_crit(Om, Or) (1 - delta), delta ~ U(0, 1e-6));
    explicit five-column parameters; z ~ logU(1e-4, 1100)."""
    rng = np.random.default_rng(seed)
    params = np.zeros((B, 5))
    z = np.zeros((B, n))
    for b in range(B):
        H0 = None
        while True:
            Om = rng.uniform(0.05, 0.6)
            Or = 10.0 ** rng.uniform(-5.0, -4.0)
            H0 = rng.uniform(60.0, 80.0)
            if b % 2 == 0:
                Ok = rng.uniform(-1e-6, 1e-6)
                OL = 1.0 - Om - Or - Ok
            else:
                delta = rng.uniform(0.0, 1e-6)
                OL = ol_critical(Om, Or) * (1.0 - delta)
                Ok = 1.0 - Om - OL - Or
            if has_big_bang(Om, OL, Or, Ok):
                break
        params[b] = (H0, Om, OL, Or, Ok)
        z[b] = 10.0 ** rng.uniform(-4.0, np.log10(1100.0), n)
    return Batch("stress-%dx%d" % (B, n), params, z.reshape(-1),
                 np.arange(B + 1, dtype=np.int64) * n)


def between_batch(B=4096, n=1024, seed=5, z1max=3.0, dzmax=10.0):
    """General limits: cosmologies as general_batch; per row a lower limit
    z1 ~ U(0, z1max) (an observer, lens or absorber redshift), then n upper
    limits z2 = z1 + dz, dz ~ U(0, dzmax).  extra["z1"] holds z1 [B]."""
    rng = np.random.default_rng(seed)
    params = np.zeros((B, 4))
    z1 = np.zeros(B)
    z = np.zeros((B, n))
    for b in range(B):
        H0, Om, OL, Or = _draw_cosmo(rng)
        params[b] = (H0, Om, OL, Or)
        z1[b] = rng.uniform(0.0, z1max)
        z[b] = z1[b] + rng.uniform(0.0, dzmax, n)
    return Batch("between-%dx%d" % (B, n), params, z.reshape(-1),
                 np.arange(B + 1, dtype=np.int64) * n, extra={"z1": z1})


def limits_batch(B=65536, seed=6):
    """Upper limit at infinity (age, horizon): cosmologies as general_batch,
    one lower limit per row, half z1 ~ U(0, 10) and half z1 ~ logU(10, 1100)."""
    rng = np.random.default_rng(seed)
    params = np.zeros((B, 4))
    z1 = np.zeros(B)
    for b in range(B):
        H0, Om, OL, Or = _draw_cosmo(rng)
        params[b] = (H0, Om, OL, Or)
        z1[b] = rng.uniform(0.0, 10.0) if b % 2 == 0 else 10.0 ** rng.uniform(1.0, np.log10(1100.0))
    return Batch("limits-%d" % B, params, np.zeros(0), np.zeros(B + 1, dtype=np.int64),
                 extra={"z1": z1})


def bhm_supernovae(N=1_000_000, seed=7, truth=(0.3, 0.7), H0=70.0, alpha=2.0, beta=3.0, sigma_mu=0.14,
                   sigma_z=0.04, mu=None):
    """Mock data of the Sec. 4 supernova model: latent z ~ Gamma(alpha, rate
    beta), observed zhat ~ N(z, (1+z)^2 sigma_z^2), observed distance modulus
    muhat ~ N(mu(z), sigma_mu^2) for a radiationless cosmology (Om, OL) =
    truth.  ``mu`` maps latent redshifts to distance moduli; by default the
    cosmographic series mock_mu (tests pass exact distances).  The stand-in
    for the paper's mock sets of 10^3 to 10^6 SNe."""
    rng = np.random.default_rng(seed)
    z = rng.gamma(alpha, 1.0 / beta, N)
    z = np.maximum(z, 1e-4)
    zhat = z + (1.0 + z) * sigma_z * rng.normal(size=N)
    m = mock_mu(z, H0, truth[0], truth[1], 0.0) if mu is None else mu(z)
    muhat = m + sigma_mu * rng.normal(size=N)
    params = np.array([[H0, truth[0], truth[1], 0.0]])
    return Batch("bhm-sn-%d" % N, params, z, np.array([0, N], dtype=np.int64), m_obs=muhat, M=0.0,
                 sigma=sigma_mu, extra={"z_hat": zhat, "alpha": alpha, "beta": beta, "sigma_z": sigma_z,
                                        "truth": truth, "H0": H0})
