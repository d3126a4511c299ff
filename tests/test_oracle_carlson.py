"""Pins of the oracle's Carlson integrals (eqs. 2.6-2.12) against closed
forms, identities, scipy, brute-force quadrature and principal values."""
import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

import oracle

RNG = np.random.default_rng(12345)
RF = lambda *a: oracle.carlson("rf", *a)
RJ = lambda *a: oracle.carlson("rj", *a)
RC = lambda *a: oracle.carlson("rc", *a)
RD = lambda *a: oracle.carlson("rd", *a)


def close(a, b, tol):
    a, b = np.asarray(a), np.asarray(b)
    return np.all(np.abs(a - b) <= tol * np.maximum(np.abs(b), 1e-300))


def test_equal_arguments():
    x = RNG.uniform(0.01, 100, 50)
    assert close(RF(x, x, x), x ** -0.5, 2e-15)
    assert close(RD(x, x, x), x ** -1.5, 2e-15)
    assert close(RJ(x, x, x, x), x ** -1.5, 2e-15)
    assert close(RC(x, x), x ** -0.5, 2e-15)


def test_rf_complete_and_agm():
    y = RNG.uniform(0.1, 10, 20)
    assert close(RF(0, y, y), np.pi / (2 * np.sqrt(y)), 2e-15)
    # complete integral of the first kind: K(m) = R_F(0, 1-m, 1) = pi / (2 AGM(1, sqrt(1-m)))
    for m in [0.0, 0.1, 0.5, 0.9, 0.999]:
        a, b = 1.0, np.sqrt(1 - m)
        for _ in range(40):
            a, b = 0.5 * (a + b), np.sqrt(a * b)
        assert close(RF(0, 1 - m, 1), np.pi / (2 * a), 2e-15)


def test_rc_elementary():
    x = RNG.uniform(0.01, 5, 50)
    y = RNG.uniform(0.01, 5, 50)
    lt, gt = x < y, x > y
    ref = np.empty_like(x)
    ref[lt] = np.arccos(np.sqrt(x[lt] / y[lt])) / np.sqrt(y[lt] - x[lt])
    ref[gt] = np.arccosh(np.sqrt(x[gt] / y[gt])) / np.sqrt(x[gt] - y[gt])
    assert close(RC(x, y).real, ref, 1e-13)


def test_homogeneity_and_symmetry():
    x, y, z, p = RNG.uniform(0.1, 5, (4, 40))
    lam = RNG.uniform(0.1, 10, 40)
    assert close(RF(lam * x, lam * y, lam * z), lam ** -0.5 * RF(x, y, z), 3e-15)
    assert close(RJ(lam * x, lam * y, lam * z, lam * p), lam ** -1.5 * RJ(x, y, z, p), 3e-15)
    assert close(RC(lam * x, lam * y), lam ** -0.5 * RC(x, y), 3e-15)
    assert close(RF(y, z, x), RF(x, y, z), 3e-15) and close(RF(z, x, y), RF(x, y, z), 3e-15)
    assert close(RJ(y, z, x, p), RJ(x, y, z, p), 3e-15) and close(RJ(z, y, x, p), RJ(x, y, z, p), 3e-15)


def test_rd_cyclic_sum():
    x, y, z = RNG.uniform(0.1, 5, (3, 40))
    s = RD(x, y, z) + RD(y, z, x) + RD(z, x, y)
    assert close(s, 3 / np.sqrt(x * y * z), 3e-15)


def test_scipy_cross_check_real_and_conjugate_pair():
    x, y, z, p = RNG.uniform(0.01, 50, (4, 500))
    assert close(RF(x, y, z), sp.elliprf(x, y, z), 2e-15)
    assert close(RJ(x, y, z, p), sp.elliprj(x, y, z, p), 5e-15)
    assert close(RD(x, y, z), sp.elliprd(x, y, z), 5e-15)
    assert close(RC(x, y), sp.elliprc(x, y), 2e-15)
    c = RNG.uniform(-5, 5, 200) + 1j * RNG.uniform(0.1, 5, 200)
    a = RNG.uniform(0.01, 10, 200)
    w = RNG.uniform(0.01, 10, 200)
    assert close(RF(a, c, np.conj(c)), sp.elliprf(a, c, np.conj(c)), 3e-15)
    assert close(RJ(a, c, np.conj(c), w), sp.elliprj(a, c, np.conj(c), w), 1e-14)
    assert close(RD(c, np.conj(c), a), sp.elliprd(c, np.conj(c), a), 1e-14)
    assert close(RD(a, np.conj(c), c), sp.elliprd(a, np.conj(c), c), 1e-14)


def _brute(f):
    # int_0^inf f(t) dt with t = s/(1-s)
    g = lambda s: f(s / (1 - s)) / (1 - s) ** 2
    val, err = si.quad(g, 0, 1, epsabs=0, epsrel=1e-13, limit=500)
    return val


def test_brute_force_definitions():
    for x, y, z, p in RNG.uniform(0.2, 3, (5, 4)):
        rf = 0.5 * _brute(lambda t: 1 / np.sqrt((t + x) * (t + y) * (t + z)))
        rj = 1.5 * _brute(lambda t: 1 / ((t + p) * np.sqrt((t + x) * (t + y) * (t + z))))
        assert close(RF(x, y, z).real, rf, 1e-11)
        assert close(RJ(x, y, z, p).real, rj, 1e-11)


def _pv(f, t0):
    """(PV) int_0^inf f(t)/(t - t0) dt for t0 > 0 via QUADPACK's Cauchy weight."""
    L = 4 * t0 + 1
    a, _ = si.quad(f, 0, L, weight="cauchy", wvar=t0, epsabs=0, epsrel=1e-13, limit=500)
    b, _ = si.quad(lambda t: f(t) / (t - t0), L, np.inf, epsabs=0, epsrel=1e-13, limit=500)
    return a + b


def test_principal_values():
    for x, y, z in RNG.uniform(0.2, 3, (4, 3)):
        q = RNG.uniform(0.1, 3)
        f = lambda t: 1 / np.sqrt((t + x) * (t + y) * (t + z))
        ref = 1.5 * _pv(f, q)
        assert close(RJ(x, y, z, -q).real, ref, 1e-10)
    # conjugate pair with a real member
    a = 2.0
    c = 1.0 + 0.7j
    q = 0.8
    f = lambda t: 1 / np.sqrt(((t + a) * (t + c) * (t + np.conj(c))).real)
    assert close(RJ(a, c, np.conj(c), -q).real, 1.5 * _pv(f, q), 1e-10)
    for x in RNG.uniform(0.2, 3, 4):
        q = RNG.uniform(0.1, 3)
        ref = 0.5 * _pv(lambda t: 1 / np.sqrt(t + x), q)
        assert close(RC(x, -q).real, ref, 1e-10)


def test_principal_values_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    for x, y, z, q in RNG.uniform(0.2, 4, (6, 4)):
        ref = float(mp.re(mp.elliprj(x, y, z, -q)))
        assert close(RJ(x, y, z, -q).real, ref, 1e-13)


def _fd(f, x, h):
    return (f(x + h) - f(x - h)) / (2 * h)


def test_derivative_identities_2_10_to_2_12():
    """(2.10), (2.11) as printed; (2.12) with R_G(x1,x2,x3) in place of the
    printed R_D (the only reading consistent with finite differences), where
    6 R_G = sum_m x_m (sum_{n != m} x_n) R_D(..., x_m)."""
    for x1, x2, x3, w in RNG.uniform(0.3, 3, (6, 4)):
        h = 1e-5
        rd3 = RD(x1, x2, x3).real
        assert close(_fd(lambda v: RF(x1, x2, v).real, x3, h), -rd3 / 6, 1e-8)
        rj = RJ(x1, x2, x3, w).real
        assert close(_fd(lambda v: RJ(x1, x2, v, w).real, x3, h), 0.5 * (rj - rd3) / (w - x3), 1e-7)
        xs = [x1, x2, x3]
        rdm = [RD(x2, x3, x1).real, RD(x1, x3, x2).real, rd3]
        rg = sum(xs[m] * (sum(xs) - xs[m]) * rdm[m] for m in range(3)) / 6
        assert close(rg, sp.elliprg(x1, x2, x3), 1e-14)
        prod = np.sqrt(x1 * x2 * x3)
        d212 = 1.5 * ((w * w * RF(x1, x2, x3).real - 2 * w * rg + prod)
                      / (w * (w - x1) * (w - x2) * (w - x3))
                      - sum(1 / (w - x) for x in xs) * rj / 3)
        assert close(_fd(lambda v: RJ(x1, x2, x3, v).real, w, h), d212, 1e-7)
