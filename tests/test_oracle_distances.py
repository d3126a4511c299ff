"""Pins of the oracle's distances (O1 quadrature, O2 Carlson assembly) and
gradients (O4 Leibniz rule) against closed forms, brute force, each other and
finite differences."""
import os

import numpy as np
import pytest
import scipy.special as sp

import oracle
from paper_2212_01937_gb300 import workloads

C = 299792.458
TH = 977.7922216807891
H0 = 70.0
DH, tH = C / H0, TH / H0
ZS = np.array([1e-4, 0.01, 0.5, 1.0, 3.0, 10.0])


def rel(a, b):
    return np.max(np.abs(np.asarray(a) / np.asarray(b) - 1))


def q(p, z, **kw):
    return oracle.quad_distances(np.asarray(p, float), np.asarray(z, float), **kw)


def test_einstein_de_sitter():
    o = q([H0, 1.0, 0.0, 0.0, 0.0], ZS)
    x = 1 + ZS
    L = np.log1p(ZS)   # closed forms written without cancellation at small z
    assert rel(o[:, 0], -2 * DH * np.expm1(-0.5 * L)) < 1e-13
    assert rel(o[:, 1], -2 / 3 * tH * np.expm1(-1.5 * L)) < 1e-13
    assert rel(o[:, 2], 2 / 3 * DH * np.expm1(1.5 * L)) < 1e-13
    assert rel(o[:, 3], o[:, 0]) < 1e-15


def test_milne():
    o = q([H0, 0.0, 0.0, 0.0, 1.0], ZS)
    assert rel(o[:, 0], DH * np.log1p(ZS)) < 1e-13
    assert rel(o[:, 3], DH * ZS * (2 + ZS) / (2 * (1 + ZS))) < 1e-13
    assert rel(o[:, 1], tH * ZS / (1 + ZS)) < 1e-13
    assert rel(o[:, 2], DH * (ZS + ZS ** 2 / 2)) < 1e-13
    assert rel(o[:, 4], (1 + ZS) * o[:, 3]) < 1e-15
    assert rel(o[:, 5], 5 * np.log10(o[:, 4]) + 25) < 1e-15


def test_flat_radiationless_closed_forms():
    zs = ZS[ZS >= 0.5]   # the closed forms below are differences of two end points
    for Om in [0.1, 0.3, 0.8]:
        OL = 1 - Om
        o = q([H0, Om, OL, 0.0], zs)
        s = np.sqrt(OL / Om)
        t = 2 / (3 * np.sqrt(OL)) * tH * (np.arcsinh(s) - np.arcsinh(s * (1 + zs) ** -1.5))
        assert rel(o[:, 1], t) < 1e-13
        # int_0^x dt / sqrt(OL + Om t^3) = x 2F1(1/2, 1/3; 4/3; -(Om/OL) x^3) / sqrt(OL)
        F = lambda x: x * sp.hyp2f1(0.5, 1 / 3, 4 / 3, -(Om / OL) * x ** 3) / np.sqrt(OL)
        assert rel(o[:, 0], DH * (F(1 + zs) - F(1.0))) < 1e-13


def test_flat_matter_radiation():
    Om, Or = 0.7, 0.3
    o = q([H0, Om, 0.0, Or], ZS)
    a = 1 / (1 + ZS)
    # sqrt(Or + Om) - sqrt(Or + Om a), rationalised: Om (1 - a) / (sum of roots)
    diff = Om * (ZS / (1 + ZS)) / (np.sqrt(Or + Om) + np.sqrt(Or + Om * a))
    assert rel(o[:, 0], DH * 2 / Om * diff) < 1e-13


def test_simpson_brute_force():
    for p in ([70.0, 0.3, 0.7, 1e-5], [65.0, 0.5, 0.2, 8e-5], [75.0, 0.05, 1.1, 2e-5]):
        for z in (0.02, 1.3, 8.0):
            ref = oracle.simpson(np.array(p), z, n=200_000)
            o = q(p, [z])[0]
            assert rel(o[:3], ref) < 1e-11


def _config2_small(B=24, n=16, seed=21):
    return workloads.general_batch(B=B, n=n, seed=seed)


def test_carlson_vs_quadrature_random():
    b = _config2_small()
    zq = np.concatenate([b.z, np.full(b.B, 1100.0)])
    offs = np.concatenate([b.offsets[:-1] + np.arange(b.B), [b.nnz + b.B]])
    # interleave one z=1100 point per row
    z2 = np.concatenate([np.append(b.z[b.offsets[i]:b.offsets[i + 1]], 1100.0) for i in range(b.B)])
    o1 = q(b.params, z2, offsets=offs)
    o2, im = oracle.carlson_distances(b.params, z2, offsets=offs, return_imag=True)
    assert rel(o2[:, 0], o1[:, 0]) < 1e-13
    assert rel(o2[:, 1], o1[:, 1]) < 1e-13
    assert rel(o2[:, 2], o1[:, 2]) < 2e-10     # eq. (3.9) loses digits in FP64 (Sec. 3.2.1)
    assert np.all(np.abs(im) <= 1e-9 * np.abs(o1[:, :3]))
    assert zq.size == z2.size


def test_carlson_cubic_vs_quadrature():
    for p in ([70.0, 0.3, 0.7, 0.0], [60.0, 0.05, 0.2, 0.0], [80.0, 0.6, 1.1, 0.0], [70.0, 0.4, 0.3, 0.0]):
        z = np.array([1e-3, 0.3, 2.0, 10.0, 1100.0])
        o1, o2 = q(p, z), oracle.carlson_distances(np.array(p), z)
        assert rel(o2[:, :2], o1[:, :2]) < 1e-13
        assert rel(o2[:, 2], o1[:, 2]) < 1e-11    # (B.3) also loses a few digits at high z


def test_fig2_setups_mpmath():
    """Sec. 3.2.1 / Fig. 2 setups against mpmath quadrature at 30 digits."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    for Or in (0.0, 1e-5):
        p = [70.0, 0.3, 0.7, Or]
        Ok = 1 - 0.3 - 0.7 - Or
        for z in (1e-3, 0.1, 1.0, 10.0, 1000.0):
            Q = lambda a: Or + 0.3 * a + Ok * a ** 2 + 0.7 * a ** 4
            a0 = 1 / (1 + mp.mpf(z))
            ref = [mp.quad(lambda a: 1 / mp.sqrt(Q(a)), [a0, 1]) * DH,
                   mp.quad(lambda a: a / mp.sqrt(Q(a)), [a0, 1]) * tH,
                   mp.quad(lambda a: a ** -2 / mp.sqrt(Q(a)), [a0, 1]) * DH]
            o = q(p, [z])[0]
            assert rel(o[:3], np.array([float(v) for v in ref])) < 1e-13


def test_fig2_golden_file():
    """Stored O1 values for the Fig. 2 setups (written by tests/golden/make_golden.py)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "fig2_setups.txt")
    data = np.loadtxt(path)
    for Or in (0.0, 1e-5):
        rows = data[data[:, 0] == Or]
        o = q([70.0, 0.3, 0.7, Or], rows[:, 1])
        assert rel(o[:, :3], rows[:, 2:5]) < 1e-14


def test_zero_redshift_and_monotonic():
    b = _config2_small(B=6, n=1)
    z = np.linspace(0.0, 5.0, 41)
    for p in b.params:
        o = q(p, z)
        assert np.all(o[0, :5] == 0.0) and o[0, 5] == -np.inf
        assert np.all(np.diff(o[:, 0]) > 0) and np.all(np.diff(o[:, 1]) > 0)


def test_gradients_vs_finite_differences():
    b = _config2_small(B=5, n=4, seed=33)
    for ncol in (4, 5):
        params = b.params if ncol == 4 else np.column_stack(
            [b.params, 1 - b.params[:, 1:4].sum(axis=1)])
        o, J = q(params, b.z, offsets=b.offsets, grad=True)
        for k in range(ncol):
            h = 1e-5 * max(abs(params[:, k]).max(), 1e-3) if k else 1e-4
            if k == 3:
                h = 1e-7
            pp, pm = params.copy(), params.copy()
            pp[:, k] += h
            pm[:, k] -= h
            fd = (q(pp, b.z, offsets=b.offsets) - q(pm, b.z, offsets=b.offsets)) / (2 * h)
            err = np.abs(J[:, :, k] - fd) / np.maximum(np.abs(fd), 1e-6 * np.abs(o))
            assert err.max() < 1e-6, (ncol, k, err.max())
        # H0 invariants
        assert rel(J[:, :5, 0], -o[:, :5] / params[b.offsets[:-1].searchsorted(np.arange(b.nnz), 'right') - 1, 0:1]) < 1e-14
        assert np.allclose(J[:, 5, 0] * params[np.repeat(np.arange(b.B), 4), 0], -5 / np.log(10), rtol=1e-14)


def test_curvature_map_small_curvature():
    """Near flatness the curvature map uses its Taylor series; its value and
    its Ok derivative must agree with finite differences of the sinh/sin form
    evaluated away from the switch."""
    z = np.array([0.3, 1.0, 3.0])
    for Ok in (3e-3, -3e-3, 1e-6, -1e-6, 0.0):
        p = np.array([70.0, 0.3, 0.7 - Ok - 1e-5, 1e-5, Ok])
        o, J = q(p, z, grad=True)
        D = o[:, 0] / DH
        if Ok > 0:
            S = np.sinh(np.sqrt(Ok) * D) / np.sqrt(Ok)
        elif Ok < 0:
            S = np.sin(np.sqrt(-Ok) * D) / np.sqrt(-Ok)
        else:
            S = D
        assert rel(o[:, 3], DH * S) < 1e-14
        h = 1e-4
        pp, pm = p.copy(), p.copy()
        pp[4] += h
        pm[4] -= h
        fd = (q(pp, z)[:, 3] - q(pm, z)[:, 3]) / (2 * h)
        assert rel(J[:, 3, 4], fd) < 1e-6


def test_near_boundary_peak_resolved():
    """Near the no-Big-Bang boundary (Sec. 3, Fig. 1) the integrand 1/E has a
    narrow peak at the complex pair's real part; the quadrature must resolve
    it.  Pinned against mpmath quadrature split at the peak and against the
    Carlson assembly (which is exact there, fn14's branch caveat aside)."""
    p = np.array([68.6741596, 0.286697693, 1.69305727, 9.52482287e-05, -0.979850211])
    z = np.array([0.5, 1.3, 2.0, 10.0, 525.0])
    o1 = q(p, z)
    o2 = oracle.carlson_distances(p, z)
    assert rel(o2[:, :2], o1[:, :2]) < 1e-12
    assert rel(o2[:, 2], o1[:, 2]) < 2e-11   # (3.9) as printed (see test_x_cancellation_as_printed)
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    Om, OL, Or, Ok = [mp.mpf(float(x)) for x in p[1:]]
    E = lambda zz: mp.sqrt(Or * (1 + zz) ** 4 + Om * (1 + zz) ** 3 + Ok * (1 + zz) ** 2 + OL)
    zp = mp.mpf(1.2761806)
    dh = 299792.458 / p[0]
    for zi, oi in zip(z, o1):
        pts = [0] + [x for x in (zp - 0.05, zp - 0.005, zp, zp + 0.005, zp + 0.05) if x < zi] + [mp.mpf(zi)]
        ref = float(mp.quad(lambda zz: 1 / E(zz), pts)) * dh
        # Q(a) at the peak is ~1e-6 of its terms; the compensated evaluation
        # of Q keeps the integrand's relative accuracy there
        assert abs(oi[0] / ref - 1) < 1e-13


def test_stress_rows_quadrature_vs_carlson():
    s = workloads.precision_stress(B=6, n=25, seed=4)
    o1 = q(s.params, s.z, offsets=s.offsets)
    o2 = oracle.carlson_distances(s.params, s.z, offsets=s.offsets)
    assert rel(o2[:, :2], o1[:, :2]) < 1e-12


def test_stress_boundary_vs_mpmath_quadrature():
    """Cosmologies within 1e-6 of the no-Big-Bang boundary (config-5 draws):
    d_C, t and X of O1 and O2 against 34-digit quadrature of the defining
    integrals (2.3)-(2.5) in the scale factor, split at the minimum of Q(a)
    and at multiples of its peak width.  The FP64 parameters are exact
    inputs; the integrals of the polynomial they define are computed here
    without rounding, so this bounds the oracles' own error on the set."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 34
    s = workloads.precision_stress(B=12, n=3, seed=4)
    sel = np.arange(1, 12, 2)                     # the near-boundary half
    P = s.params[sel]
    Z = s.z.reshape(12, 3)[sel]
    Z[:, 0] = [1.35, 4.5, 30.0, 120.0, 0.9, 700.0]
    o1 = q(P, Z.reshape(-1), offsets=np.arange(7) * 3)
    o2 = oracle.carlson_distances(P, Z.reshape(-1), offsets=np.arange(7) * 3)
    for b in range(P.shape[0]):
        H0, Om, OL, Or, Ok = [mp.mpf(float(x)) for x in P[b]]
        Q = lambda a: Or + Om * a + Ok * a * a + OL * a ** 4
        amin = mp.findroot(lambda a: Om + 2 * Ok * a + 4 * OL * a ** 3, 0.45)
        w = mp.sqrt(Q(amin) / (Ok + 6 * OL * amin ** 2))
        for j in range(3):
            a0 = 1 / (1 + mp.mpf(float(Z[b, j])))
            pts = [a0] + sorted(amin + k * w for k in (-100, -10, -1, 0, 1, 10, 100)
                                if a0 < amin + k * w < 1) + [mp.mpf(1)]
            ref = [mp.quad(lambda a: wt(a) / mp.sqrt(Q(a)), pts) for wt in (lambda a: 1, lambda a: a,
                                                                            lambda a: 1 / a ** 2)]
            ref = np.array([float(ref[0]) * 299792.458 / float(H0), float(ref[1]) * 977.7922216807891 / float(H0),
                            float(ref[2]) * 299792.458 / float(H0)])
            i = 3 * b + j
            assert np.all(np.abs(o1[i, :3] / ref - 1) < 1e-12), (b, j, o1[i, :3] / ref - 1)
            assert np.all(np.abs(o2[i, :2] / ref[:2] - 1) < 1e-12), (b, j, o2[i, :3] / ref - 1)
