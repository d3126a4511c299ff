"""Pins of the oracle's roots (eq. 3.2) and their App. A derivatives."""
import numpy as np
import pytest

import oracle
from paper_2212_01937_gb300 import workloads


def _batch():
    b = workloads.general_batch(B=40, n=1, seed=7)
    extra = np.array([[70, 0.3, 0.7, 0.0], [70, 0.3, 0.7, 1e-5], [60, 0.05, 0.2, 0.0],
                      [70, 0.6, 1.1, 5e-5], [70, 0.2, 0.06, 2.4e-5]])
    return np.vstack([b.params, extra])


def test_vieta_and_residual():
    P = _batch()
    rho, nroot = oracle.roots_x(P)
    coef = oracle.poly_coeffs_x(P)
    for b in range(P.shape[0]):
        m = nroot[b]
        r = rho[b, :m]
        rebuilt = coef[b, m] * np.poly(r)[::-1]              # lowest power first
        assert np.allclose(rebuilt.real, coef[b, :m + 1], rtol=1e-13, atol=1e-13 * np.abs(coef[b]).max())
        assert np.all(np.abs(rebuilt.imag) <= 1e-12 * np.abs(coef[b]).max())
        res = np.abs(np.polyval(coef[b, :m + 1][::-1], r))
        bound = 8 * np.finfo(float).eps * sum(abs(coef[b, k]) * np.abs(r) ** k for k in range(m + 1))
        assert np.all(res <= bound)


def test_roots_vs_mpmath_polyroots():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    P = _batch()
    rho, nroot = oracle.roots_x(P)
    coef = oracle.poly_coeffs_x(P)
    for b in range(P.shape[0]):
        m = nroot[b]
        ref = mp.polyroots([mp.mpf(c) for c in coef[b, :m + 1][::-1]], maxsteps=400, extraprec=300)
        ref = np.array([complex(x) for x in ref])
        for r in rho[b, :m]:
            k = np.argmin(np.abs(ref - r))
            assert abs(ref[k] - r) <= 4e-15 * max(abs(ref[k]), 1.0)


def test_appendix_a_jacobian():
    P = _batch()
    rho, nroot = oracle.roots_x(P)
    for b in range(P.shape[0]):
        m = nroot[b]
        r = rho[b, :m]
        D = oracle.root_coef_jacobian(r)
        # closed form of (A.2) evaluated at z = r_j: d r_j / d c_i = -r_j^i / prod_{k != j}(r_j - r_k)
        for j in range(m):
            den = np.prod([r[j] - r[k] for k in range(m) if k != j])
            ref = np.array([-r[j] ** i / den for i in range(m)])
            # C spans ~1e12 in scale when Or ~ 1e-5 (big root ~ -Om/Or): the solve of
            # (A.4) is accurate to cond(C) eps relative to the column's largest entry
            assert np.all(np.abs(D[:, j] - ref) <= 1e-9 * np.abs(ref).max()), (b, j)


def test_param_jacobian_vs_finite_differences():
    P = _batch()[:12]
    rho, nroot = oracle.roots_x(P)
    J = oracle.root_param_jacobian(P, rho, nroot)
    for k, h in ((1, 1e-7), (2, 1e-7), (3, 1e-10)):
        pp, pm = P.copy(), P.copy()
        pp[:, k] += h
        pm[:, k] -= h
        rp, _ = oracle.roots_x(pp)
        rm, _ = oracle.roots_x(pm)
        for b in range(P.shape[0]):
            m = nroot[b]
            if m == 3 and k == 3:
                continue
            for j in range(m):
                # match roots by proximity (ordering may change)
                ip = np.argmin(np.abs(rp[b, :m] - rho[b, j]))
                im = np.argmin(np.abs(rm[b, :m] - rho[b, j]))
                fd = (rp[b, ip] - rm[b, im]) / (2 * h)
                assert abs(J[b, j, k - 1] - fd) <= 2e-5 * max(abs(fd), 1.0), (b, j, k)


def test_physicality_classification_agrees_with_q_min():
    rng = np.random.default_rng(3)
    for _ in range(300):
        Om, OL, Or = rng.uniform(-0.2, 1.0), rng.uniform(-0.5, 3.0), 10 ** rng.uniform(-6, -3)
        rho, nroot = oracle.roots_x(np.array([[70, Om, OL, Or]]))
        _, nobb = oracle.classify_roots(rho, nroot)
        assert nobb[0] == (not workloads.has_big_bang(Om, OL, Or))


def test_near_double_roots_to_the_last_bit():
    """Near the no-Big-Bang boundary (Fig. 1) two roots of E^2 nearly coincide
    (config-5 draws: delta <= 1e-6, pair separation ~1e-3): the polished
    roots must still be those of the stated FP64 polynomial to within one
    rounding of each part (40-digit mpmath polyroots), since the distances'
    sensitivity to the pair's imaginary part grows like its inverse."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    s = workloads.precision_stress(B=40, n=1, seed=4)
    P = s.params[1::2]
    rho, nroot = oracle.roots_x(P)
    coef = oracle.poly_coeffs_x(P)
    for b in range(P.shape[0]):
        ref = mp.polyroots([mp.mpf(float(c)) for c in coef[b, ::-1]], maxsteps=400, extraprec=400)
        for r in ref:
            rr, ri = float(mp.re(r)), float(mp.im(r))
            j = np.argmin(np.abs(rho[b] - complex(rr, ri)))
            assert abs(rho[b, j].real - rr) <= np.spacing(abs(rr)), (b, rho[b, j], r)
            assert abs(rho[b, j].imag - ri) <= np.spacing(abs(ri)) + 1e-300, (b, rho[b, j], r)
