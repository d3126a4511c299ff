"""Pins of the oracle with the further components the method allows (fn4):
w = -1/3 (density Os, scaling as (1+z)^2 like curvature but outside the
curvature map) and w = -2/3 (Ox, scaling as (1+z)); parameter rows
(H0, Om, OL, Or, Ok, Os, Ox), every density explicit."""
import numpy as np

import oracle

C = 299792.458
TH = 977.7922216807891
H0 = 70.0
DH, tH = C / H0, TH / H0
Z = np.array([1e-3, 0.1, 0.5, 1.0, 3.0, 10.0])


def rel(a, b):
    return np.max(np.abs(np.asarray(a) / np.asarray(b) - 1))


def test_zero_extra_components_reproduce_five_columns():
    p5 = np.array([[70.0, 0.3, 0.6, 5e-5, 0.1 - 5e-5], [65.0, 0.2, 0.9, 2e-5, -0.1 - 2e-5],
                   [72.0, 0.3, 0.7, 0.0, 0.0]])
    p7 = np.column_stack([p5, np.zeros((3, 2))])
    z = np.tile(Z, 3)
    offs = np.arange(4) * Z.size
    o5, J5 = oracle.quad_distances(p5, z, offs, grad=True)
    o7, J7 = oracle.quad_distances(p7, z, offs, grad=True)
    assert np.array_equal(o5, o7) and np.array_equal(J5, J7[:, :, :5])
    assert np.array_equal(oracle.carlson_distances(p5, z, offs), oracle.carlson_distances(p7, z, offs))


def test_pure_components_closed_forms():
    x = 1 + Z
    # w = -2/3 alone: E^2 = 1 + z
    o = oracle.quad_distances([H0, 0, 0, 0, 0, 0, 1.0], Z)
    assert rel(o[:, 0], 2 * DH * (np.sqrt(x) - 1)) < 1e-12
    assert rel(o[:, 1], 2 * tH * (1 - x ** -0.5)) < 1e-12
    assert rel(o[:, 2], 0.4 * DH * (x ** 2.5 - 1)) < 1e-12
    # w = -1/3 alone: E^2 = (1+z)^2, spatially flat (d_M = chi, unlike Milne's sinh)
    o = oracle.quad_distances([H0, 0, 0, 0, 0, 1.0, 0], Z)
    assert rel(o[:, 0], DH * np.log1p(Z)) < 1e-13
    assert rel(o[:, 1], tH * Z / x) < 1e-13
    assert rel(o[:, 2], DH * (Z + Z ** 2 / 2)) < 1e-13
    assert rel(o[:, 3], o[:, 0]) < 1e-15


def _mixtures():
    return np.array([[70.0, 0.3, 0.6, 5e-5, 0.05, 0.03, 0.02 - 5e-5],
                     [68.0, 0.25, 0.5, 8e-5, -0.05, 0.2, 0.1 - 8e-5],
                     [72.0, 0.4, 0.7, 3e-5, 0.0, -0.05, -0.05 - 3e-5],
                     [70.0, 0.3, 0.6, 0.0, 0.0, 0.05, 0.05],
                     [66.0, 0.2, 0.8, 0.0, -0.1, 0.08, 0.02]])


def test_carlson_vs_quadrature_with_components():
    """Eqs. (3.7)-(3.9) / (B.1)-(B.3) hold for any quartic / cubic: with the
    extra components only the roots change."""
    P = _mixtures()
    z = np.tile(np.append(Z, 1100.0), P.shape[0])
    offs = np.arange(P.shape[0] + 1) * (Z.size + 1)
    o1 = oracle.quad_distances(P, z, offs)
    o2, im = oracle.carlson_distances(P, z, offs, return_imag=True)
    assert rel(o2[:, :2], o1[:, :2]) < 1e-12
    assert rel(o2[:, 2], o1[:, 2]) < 1e-9
    assert np.all(np.abs(im) <= 1e-9 * np.abs(o1[:, :3]))
    # general limits and the age as well
    z1 = np.array([0.5, 1.0, 0.0, 2.0, 0.3])
    zb = np.concatenate([z1[i] + np.array([0.01, 1.0, 20.0]) for i in range(P.shape[0])])
    ob = np.arange(P.shape[0] + 1) * 3
    assert rel(oracle.carlson_between(P, z1, zb, ob)[:, :2], oracle.quad_between(P, z1, zb, ob)[:, :2]) < 1e-12
    assert rel(oracle.carlson_limits(P, z1), oracle.quad_limits(P, z1)) < 1e-12


def test_component_gradients():
    """Leibniz-rule derivatives w.r.t. Os and Ox against central differences;
    Os enters E^2 exactly as Ok does, so d chi / d Os = d chi / d Ok, while
    d_M differs by the curvature map's own dependence on Ok."""
    P = _mixtures()[:3]
    z = np.tile(Z, P.shape[0])
    offs = np.arange(P.shape[0] + 1) * Z.size
    o, J = oracle.quad_distances(P, z, offs, grad=True)
    for k in (5, 6):
        h = 1e-6
        pp, pm = P.copy(), P.copy()
        pp[:, k] += h
        pm[:, k] -= h
        fd = (oracle.quad_distances(pp, z, offs) - oracle.quad_distances(pm, z, offs)) / (2 * h)
        err = np.abs(J[:, :, k] - fd) / np.maximum(np.abs(fd), 1e-6 * np.abs(o))
        assert err.max() < 1e-6, (k, err.max())
    assert np.array_equal(J[:, :3, 5], J[:, :3, 4])
    assert not np.allclose(J[:, 3, 5], J[:, 3, 4], rtol=1e-3)
