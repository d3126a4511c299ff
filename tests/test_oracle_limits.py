"""Pins of the oracle with general limits (eqs. 2.3-2.5 from z1 to z2, and
z2 -> infinity: the age t(z1, inf) and the comoving horizon chi(z1, inf)),
against closed forms, additivity of the integrals, the quadrature and finite
differences."""
import numpy as np

import oracle
from paper_2212_01937_gb300 import workloads

C = 299792.458
TH = 977.7922216807891
H0 = 70.0
DH, tH = C / H0, TH / H0
Z1 = np.array([0.0, 0.01, 0.3, 1.0, 2.5, 7.0])


def rel(a, b):
    return np.max(np.abs(np.asarray(a) / np.asarray(b) - 1))


def _pairs(z1s, dzs):
    """One row per z1, the same dz offsets in every row."""
    z2 = np.concatenate([z + dzs for z in z1s])
    return z2, np.arange(len(z1s) + 1, dtype=np.int64) * len(dzs)


DZ = np.array([1e-3, 0.05, 0.7, 3.0, 40.0])


def test_milne_between():
    z2, offs = _pairs(Z1, DZ)
    z1 = np.repeat(Z1, DZ.size)
    p = np.tile([H0, 0.0, 0.0, 0.0, 1.0], (Z1.size, 1))
    o = oracle.quad_between(p, Z1, z2, offsets=offs)
    x1, x2 = 1 + z1, 1 + z2
    assert rel(o[:, 0], DH * np.log(x2 / x1)) < 1e-12
    assert rel(o[:, 1], tH * (z2 - z1) / (x1 * x2)) < 1e-13
    assert rel(o[:, 2], DH * (z2 - z1) * (1 + (z1 + z2) / 2)) < 1e-13
    assert rel(o[:, 3], DH * (z2 - z1) * (x1 + x2) / (2 * x1 * x2)) < 1e-12   # sinh(ln(x2/x1))
    assert rel(o[:, 4], x2 / x1 ** 2 * o[:, 3]) < 1e-15


def test_einstein_de_sitter_between():
    z2, offs = _pairs(Z1, DZ)
    z1 = np.repeat(Z1, DZ.size)
    p = np.tile([H0, 1.0, 0.0, 0.0, 0.0], (Z1.size, 1))
    o = oracle.quad_between(p, Z1, z2, offsets=offs)
    x1, x2 = 1 + z1, 1 + z2
    # differences of powers written as x1^k expm1(k log(x2/x1)), without cancellation
    L = np.log1p((z2 - z1) / x1)
    assert rel(o[:, 0], -2 * DH * x1 ** -0.5 * np.expm1(-0.5 * L)) < 1e-12
    assert rel(o[:, 1], -2 / 3 * tH * x1 ** -1.5 * np.expm1(-1.5 * L)) < 1e-12
    assert rel(o[:, 2], 2 / 3 * DH * x1 ** 1.5 * np.expm1(1.5 * L)) < 1e-12


def test_closed_form_ages_and_horizons():
    x1 = 1 + Z1
    # Einstein-de Sitter
    o = oracle.quad_limits(np.tile([H0, 1.0, 0.0, 0.0, 0.0], (Z1.size, 1)), Z1)
    assert rel(o[:, 0], 2 * DH * x1 ** -0.5) < 1e-13
    assert rel(o[:, 1], 2 / 3 * tH * x1 ** -1.5) < 1e-13
    # Milne: age 1/(H0 (1+z)) (the horizon diverges)
    o = oracle.quad_limits(np.tile([H0, 0.0, 0.0, 0.0, 1.0], (Z1.size, 1)), Z1)
    assert rel(o[:, 1], tH / x1) < 1e-13
    # flat radiationless: age (2 / (3 H0 sqrt(OL))) asinh(sqrt(OL/Om) (1+z)^-3/2)
    for Om in (0.1, 0.3, 0.8):
        OL = 1 - Om
        o = oracle.quad_limits(np.tile([H0, Om, OL, 0.0], (Z1.size, 1)), Z1)
        age = 2 / (3 * np.sqrt(OL)) * tH * np.arcsinh(np.sqrt(OL / Om) * x1 ** -1.5)
        assert rel(o[:, 1], age) < 1e-13
    # matter + radiation only (OL = Ok = 0, explicit columns): Q(a) = Or + Om a, u = Or + Om a,
    #   chi = (2/Om)(sqrt(u) - sqrt(Or)),  t = [(2/3) u^3/2 - 2 Or u^1/2]_{Or}^{u} / Om^2
    for Om, Or in ((0.3, 1e-4), (1.0 - 5e-5, 5e-5)):
        o = oracle.quad_limits(np.tile([H0, Om, 0.0, Or, 0.0], (Z1.size, 1)), Z1)
        u = Or + Om / x1
        F = lambda v: 2 / 3 * v ** 1.5 - 2 * Or * v ** 0.5
        assert rel(o[:, 0], DH * 2 / Om * (np.sqrt(u) - np.sqrt(Or))) < 1e-12
        assert rel(o[:, 1], tH * (F(u) - F(Or)) / Om ** 2) < 1e-12


def _rows(B=12, seed=41):
    b = workloads.between_batch(B=B, n=6, seed=seed, z1max=4.0, dzmax=30.0)
    return b, b.extra["z1"]


def test_quadrature_additive():
    """chi, t, d_abs are integrals: F(0, z2) = F(0, z1) + F(z1, z2)."""
    b, z1 = _rows()
    o12 = oracle.quad_between(b.params, z1, b.z, offsets=b.offsets)
    o02 = oracle.quad_distances(b.params, b.z, offsets=b.offsets)
    o01 = oracle.quad_distances(b.params, z1, offsets=np.arange(b.B + 1))
    rows = np.repeat(np.arange(b.B), np.diff(b.offsets))
    assert rel(o01[rows, :3] + o12[:, :3], o02[:, :3]) < 1e-13


def test_carlson_between_vs_quadrature():
    b, z1 = _rows()
    o1 = oracle.quad_between(b.params, z1, b.z, offsets=b.offsets)
    o2, im = oracle.carlson_between(b.params, z1, b.z, offsets=b.offsets, return_imag=True)
    assert rel(o2[:, 0], o1[:, 0]) < 1e-12
    assert rel(o2[:, 1], o1[:, 1]) < 1e-12
    assert rel(o2[:, 2], o1[:, 2]) < 2e-10   # eq. (3.9) loses digits in FP64
    assert rel(o2[:, 3:5], o1[:, 3:5]) < 1e-12
    assert np.all(np.abs(im) <= 1e-9 * np.abs(o1[:, :3]))
    # cubic (B.1)-(B.3)
    pc = np.array([[70.0, 0.3, 0.7, 0.0], [60.0, 0.05, 0.2, 0.0], [80.0, 0.6, 1.1, 0.0]])
    z1c = np.array([0.4, 2.0, 0.05])
    z2c = np.concatenate([z + DZ for z in z1c])
    offs = np.arange(4, dtype=np.int64) * DZ.size
    o1 = oracle.quad_between(pc, z1c, z2c, offsets=offs)
    o2 = oracle.carlson_between(pc, z1c, z2c, offsets=offs)
    assert rel(o2[:, :2], o1[:, :2]) < 1e-12
    assert rel(o2[:, 2], o1[:, 2]) < 1e-10


def test_carlson_between_reduces_to_z1_zero():
    b, _ = _rows()
    o_a = oracle.carlson_between(b.params, np.zeros(b.B), b.z, offsets=b.offsets)
    o_b = oracle.carlson_distances(b.params, b.z, offsets=b.offsets)
    assert np.array_equal(o_a, o_b)


def test_carlson_limits_vs_quadrature_and_differences():
    b = workloads.limits_batch(B=16, seed=43)
    z1 = b.extra["z1"]
    o1 = oracle.quad_limits(b.params, z1)
    o2, im = oracle.carlson_limits(b.params, z1, return_imag=True)
    assert rel(o2, o1) < 1e-12
    assert np.all(np.abs(im) <= 1e-9 * np.abs(o1))
    # t(z1, z2) = t(z1, inf) - t(z2, inf) at moderate z2 (no cancellation to speak of)
    z2 = z1 * 1.5 + 0.5
    tb = oracle.carlson_between(b.params, z1, z2, offsets=np.arange(b.B + 1))[:, 1]
    t2 = oracle.carlson_limits(b.params, z2)[:, 1]
    assert rel(o2[:, 1] - t2, tb) < 1e-10
    # cubic limits
    pc = np.array([[70.0, 0.3, 0.7, 0.0], [60.0, 0.05, 0.2, 0.0], [80.0, 0.6, 1.1, 0.0]])
    zc = np.array([0.0, 3.0, 500.0])
    assert rel(oracle.carlson_limits(pc, zc), oracle.quad_limits(pc, zc)) < 1e-12


def test_short_interval_limit():
    """chi(z1, z1 + h) -> h c / (H0 E(z1)) as h -> 0 (first order in h)."""
    b, z1 = _rows(B=6)
    h = 1e-6
    o = oracle.carlson_between(b.params, z1, z1 + h, offsets=np.arange(b.B + 1))
    Om, OL, Or = b.params[:, 1], b.params[:, 2], b.params[:, 3]
    Ok = 1 - Om - OL - Or
    x = 1 + z1
    E = np.sqrt(Or * x ** 4 + Om * x ** 3 + Ok * x ** 2 + OL)
    assert rel(o[:, 0], h * C / b.params[:, 0] / E) < 1e-5


def test_gradients_between_and_limits_vs_finite_differences():
    b, z1 = _rows(B=5, seed=45)
    for ncol in (4, 5):
        params = b.params if ncol == 4 else np.column_stack([b.params, 1 - b.params[:, 1:4].sum(axis=1)])
        o, J = oracle.quad_between(params, z1, b.z, offsets=b.offsets, grad=True)
        ol, Jl = oracle.quad_limits(params, z1, grad=True)
        for k in range(ncol):
            h = 1e-5 * max(abs(params[:, k]).max(), 1e-3) if k else 1e-4
            if k == 3:
                h = 1e-7
            pp, pm = params.copy(), params.copy()
            pp[:, k] += h
            pm[:, k] -= h
            fd = (oracle.quad_between(pp, z1, b.z, offsets=b.offsets)
                  - oracle.quad_between(pm, z1, b.z, offsets=b.offsets)) / (2 * h)
            err = np.abs(J[:, :, k] - fd) / np.maximum(np.abs(fd), 1e-6 * np.abs(o))
            assert err.max() < 1e-6, (ncol, k, err.max())
            if k == 3:   # the horizon's Or derivative varies on the scale of Or itself
                h = 2e-9
                pp, pm = params.copy(), params.copy()
                pp[:, k] += h
                pm[:, k] -= h
            fdl = (oracle.quad_limits(pp, z1) - oracle.quad_limits(pm, z1)) / (2 * h)
            errl = np.abs(Jl[:, :, k] - fdl) / np.maximum(np.abs(fdl), 1e-6 * np.abs(ol))
            assert errl.max() < 1e-6, (ncol, k, errl.max())


def test_empty_and_reversed_intervals():
    p = np.array([[70.0, 0.3, 0.7, 5e-5]])
    o = oracle.quad_between(p, [1.0], np.array([1.0, 0.5]))
    assert np.all(o[0, :5] == 0.0) and o[0, 5] == -np.inf
    assert np.all(np.isnan(o[1]))
    o2 = oracle.carlson_between(p, [1.0], np.array([1.0, 0.5]))
    assert np.all(o2[0, :5] == 0.0) and np.all(np.isnan(o2[1]))


def test_dmu_dz_closed_forms_and_differences():
    """d mu / dz (the integrand of eq. 2.3 through the curvature map):
    Milne (5/ln10)(1/z + 1/(2+z)); Einstein-de Sitter from its closed form;
    central differences of the quadrature for curved cosmologies."""
    z = np.array([0.01, 0.3, 1.0, 2.5, 6.0])
    k = 5 / np.log(10)
    g = oracle.dmu_dz([H0, 0.0, 0.0, 0.0, 1.0], z)
    assert rel(g, k * (1 / z + 1 / (2 + z))) < 1e-12
    x = 1 + z
    g = oracle.dmu_dz([H0, 1.0, 0.0, 0.0, 0.0], z)
    dm = 2 * (1 - x ** -0.5)
    assert rel(g, k * (1 / x + x ** -1.5 / dm)) < 1e-12
    for p in ([70.0, 0.3, 0.7, 5e-5], [65.0, 0.2, 0.3, 8e-5], [75.0, 0.5, 1.1, 1e-5]):
        h = 1e-5 * z
        fd = (oracle.quad_distances(p, z + h)[:, 5] - oracle.quad_distances(p, z - h)[:, 5]) / (2 * h)
        assert rel(oracle.dmu_dz(p, z), fd) < 1e-8


def test_dout_dz_against_differences():
    """All six z-derivatives against central differences of the quadrature
    (the integrands of eqs. 2.3-2.5 at the upper limit, the curvature map and
    d_L = (1+z) d_M), for open, closed and flat cosmologies; and at z = 0 the
    integrands at their lower end: d chi/dz = c/H0, d t/dz = 1/H0."""
    z = np.array([0.01, 0.3, 1.0, 2.5, 6.0])
    for p in ([70.0, 0.3, 0.7, 5e-5], [65.0, 0.2, 0.3, 8e-5], [75.0, 0.5, 1.1, 1e-5], [70.0, 0.3, 0.7, 0.0]):
        h = 1e-5 * z
        fd = (oracle.quad_distances(p, z + h) - oracle.quad_distances(p, z - h)) / (2 * h)[:, None]
        assert rel(oracle.dout_dz(p, z), fd) < 1e-8, p
    d0 = oracle.dout_dz([H0, 0.3, 0.7, 5e-5], [0.0])[0]
    assert abs(d0[0] / DH - 1) < 1e-14 and abs(d0[1] / tH - 1) < 1e-14 and d0[5] == 0.0


def test_general_limits_and_age_mpmath():
    """O1 with general limits and the age against mpmath quadrature at 30
    digits (open and closed cosmologies with radiation; radiationless)."""
    mp = __import__("pytest").importorskip("mpmath")
    mp.mp.dps = 30
    for p in ([70.0, 0.3, 0.7, 5e-5], [68.0, 0.45, 0.3, 8e-5], [72.0, 0.2, 1.0, 2e-5], [70.0, 0.3, 0.7, 0.0]):
        Om, OL, Or = (mp.mpf(v) for v in p[1:4])
        Ok = 1 - Om - OL - Or
        Q = lambda a: Or + Om * a + Ok * a ** 2 + OL * a ** 4
        DHm, tHm = mp.mpf(C) / p[0], mp.mpf(977.7922216807891) / p[0]
        for z1, z2 in ((0.2, 0.25), (1.0, 4.0), (3.0, 1100.0)):
            a1, a2 = 1 / (1 + mp.mpf(z1)), 1 / (1 + mp.mpf(z2))
            ref = [DHm * mp.quad(lambda a: 1 / mp.sqrt(Q(a)), [a2, a1]),
                   tHm * mp.quad(lambda a: a / mp.sqrt(Q(a)), [a2, a1]),
                   DHm * mp.quad(lambda a: a ** -2 / mp.sqrt(Q(a)), [a2, a1])]
            o = oracle.quad_between(p, [z1], np.array([z2]))[0]
            assert rel(o[:3], np.array([float(v) for v in ref])) < 1e-13, (p, z1, z2)
        for z1 in (0.0, 2.0, 50.0):
            a1 = 1 / (1 + mp.mpf(z1))
            # in s = sqrt(a): the integrands stay bounded at a = 0 for the radiationless case too
            age = tHm * mp.quad(lambda s: 2 * s ** 3 / mp.sqrt(Q(s * s)), [0, mp.sqrt(a1)])
            hor = DHm * mp.quad(lambda s: 2 * s / mp.sqrt(Q(s * s)), [0, mp.sqrt(a1)])
            o = oracle.quad_limits(p, [z1])[0]
            assert rel(o, np.array([float(hor), float(age)])) < 1e-13, (p, z1)
