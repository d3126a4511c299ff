"""Pins of the speed-study comparators (Sec. 3.2.2, Fig. 3): the Legendre
form of App. B.2 (eqs. B.4-B.7) and the hypergeometric flat radiationless
distance, against the quadrature oracle and against mpmath's 2F1."""
import numpy as np
import pytest

import oracle

Z = np.logspace(-3, 3, 25)


def test_legendre_form_matches_quadrature():
    """The Fig. 2 / Fig. 3 setups (flat 0.3/0.7 with and without Omega_r0 =
    1e-5) and two curved cosmologies: d_C and t in Legendre's form agree with
    the defining integrals (the form differences F~ at the two limits, which
    costs a few digits at low z, fn19)."""
    P = np.array([[70, 0.3, 0.7, 0.0], [70, 0.3, 0.7, 1e-5], [65, 0.25, 0.6, 3e-5], [72, 0.4, 0.5, 0.0]])
    Zs = np.tile(Z, len(P))
    off = np.arange(len(P) + 1) * Z.size
    L = oracle.legendre_distances(P, Zs, off)
    ref = oracle.quad_distances(P, Zs, off)
    assert np.all(np.isfinite(L))
    assert np.max(np.abs(L / ref[:, :2] - 1)) < 2e-12


def test_hypergeometric_flat_distance():
    ref = oracle.quad_distances(np.array([[70, 0.3, 0.7, 0.0]]), Z, np.array([0, Z.size]))
    h = oracle.hyp2f1_flat_distance(70, 0.3, Z)
    assert np.max(np.abs(h / ref[:, 0] - 1)) < 1e-12
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    w = mp.mpf(0.3) / mp.mpf(0.7)
    for z in (0.01, 0.7, 4.0, 300.0):
        x = 1 + mp.mpf(z)
        ex = (x * mp.hyp2f1(0.5, mp.mpf(1) / 3, mp.mpf(4) / 3, -w * x ** 3) - mp.hyp2f1(0.5, mp.mpf(1) / 3,
              mp.mpf(4) / 3, -w)) / mp.sqrt(mp.mpf(0.7)) * 299792.458 / 70
        assert abs(oracle.hyp2f1_flat_distance(70, 0.3, [z])[0] / float(ex) - 1) < 1e-13
