"""Identities the GPU duplication sequence is built on, checked with SciPy's
Carlson integrals (host only; no product code runs here).

* One duplication step on a triple (x1, y_a, y_b) whose pair is a conjugate
  pair or two reals, written on the pair's symmetric functions: with
  s1 = sqrt(x1), S = s_a + s_b, P = s_a s_b, lambda = s1 S + P,
    x1 + lambda = s1^2 + s1 S + P,  sigma' = S (S + 2 s1) / 4,  pi' = x1' S^2 / 4,
  and R_F / R_J of the triple are unchanged by the step (Carlson's
  duplication theorem, the paper's ref. [10]).
* R_C's partial derivatives (eq. 2.10 with R_C(x, y) = R_F(x, y, y)) and
  Euler's relation for R_F, homogeneous of degree -1/2:
    x R_D(y, y, x) + 2 y R_D(x, y, y) = 3 R_C(x, y).
"""
import numpy as np
import pytest

special = pytest.importorskip("scipy.special")
mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 30


def _pairs(rng, n):
    """Conjugate pairs (including ones close to the negative real axis) and real pairs."""
    out = []
    for _ in range(n):
        r = rng.uniform(0.1, 3.0)
        for ang in (rng.uniform(0.0, np.pi), np.pi - 10.0 ** rng.uniform(-6, -2)):
            ya = r * np.exp(1j * ang)
            out.append((ya, np.conj(ya)))
        out.append((complex(rng.uniform(0.1, 3.0)), complex(rng.uniform(0.1, 3.0))))
    return out


def test_symmetric_duplication_step():
    rng = np.random.default_rng(3)
    for ya, yb in _pairs(rng, 40):
        x1 = rng.uniform(0.1, 3.0)
        s1, sa, sb = np.sqrt(x1), np.sqrt(ya), np.sqrt(yb)          # principal roots
        S, P = (sa + sb).real, (sa * sb).real
        assert abs((sa + sb).imag) < 1e-12 and abs((sa * sb).imag) < 1e-12
        lam = s1 * S + P
        # member-wise step (Carlson's duplication)
        lam_m = s1 * sa + s1 * sb + sa * sb
        assert abs(lam - lam_m) <= 1e-12 * abs(lam_m)
        xa, ya2, yb2 = (x1 + lam) / 4, (ya + lam) / 4, (yb + lam) / 4
        # the symmetric forms, every term non-negative
        assert abs((x1 + lam) - (s1 * s1 + s1 * S + P)) <= 1e-12 * (x1 + lam)
        # (the member-wise sums cancel near the negative real axis, so they are
        # compared on the scale of their terms; the symmetric forms do not)
        sig2 = S * (S + 2 * s1) / 4
        pi2 = xa * S * S / 4
        scale = (abs(ya) + abs(yb) + 2 * abs(lam)) / 4
        assert abs((ya2 + yb2) - sig2) <= 1e-12 * scale
        assert abs(ya2 * yb2 - pi2) <= 1e-12 * scale * scale
        # the step leaves the integrals unchanged: the 30-digit values of the
        # original triple against double-precision values after the step, whose
        # arguments no longer lie near the negative real axis
        rf0 = complex(mpmath.elliprf(x1, mpmath.mpc(ya), mpmath.mpc(yb)))
        if ya.imag:   # the stepped conjugate pair from its symmetric functions
            im = np.sqrt(max(pi2 - (sig2 / 2) ** 2, 0.0)) * np.sign(ya.imag)
            ys_a, ys_b = complex(sig2 / 2, im), complex(sig2 / 2, -im)
        else:
            ys_a, ys_b = ya2, yb2
        rf1 = special.elliprf(xa, ys_a, ys_b)
        assert abs(rf0 - rf1) <= 1e-13 * abs(rf0)
        p = rng.uniform(0.2, 3.0)
        rj0 = complex(mpmath.elliprj(x1, mpmath.mpc(ya), mpmath.mpc(yb), p))
        # one step of R_J's duplication: R_J = 6 R_C(d^2, d^2 + delta) + R_J(x', y', z', p') / 4
        # with d = (sqrt p + s1)(sqrt p + s_a)(sqrt p + s_b) = (sqrt p + s1)(p + sqrt(p) S + P),
        # delta = (p - x1)(p - y_a)(p - y_b), p' = (p + lambda) / 4
        sq = np.sqrt(p)
        gp = (sq + s1) * (p + sq * S + P)
        assert abs(gp - (sq + s1) * (sq + sa) * (sq + sb)) <= 1e-12 * abs(gp)
        d = (sq + s1) * (sq + sa) * (sq + sb)
        delta = (p - x1) * (p - ya) * (p - yb)
        term = 6.0 * special.elliprc(d * d, d * d + delta)
        rj1 = special.elliprj(xa, ys_a, ys_b, (p + lam) / 4)
        assert abs(rj0 - (term + rj1 / 4)) <= 1e-12 * abs(rj0)


def test_rc_partials_euler_relation():
    rng = np.random.default_rng(5)
    for _ in range(200):
        y = 10.0 ** rng.uniform(-3, 3)
        x = y * 10.0 ** rng.uniform(-8, 8)
        rc = special.elliprc(x, y)
        rd1 = special.elliprd(y, y, x)          # x special
        rdy = special.elliprd(x, y, y)          # a pair member special
        assert abs(x * rd1 + 2 * y * rdy - 3 * rc) <= 1e-12 * 3 * rc
        # the gradient the GPU forms: dR_C/dx = -R_D(y,y,x)/6,
        # dR_C/dy = (x R_D(y,y,x) - 3 R_C) / (6 y)
        gx, gy = -rd1 / 6, (x * rd1 - 3 * rc) / (6 * y)
        hx, hy = 1e-6 * x, 1e-6 * y
        fx = (special.elliprc(x + hx, y) - special.elliprc(x - hx, y)) / (2 * hx)
        fy = (special.elliprc(x, y + hy) - special.elliprc(x, y - hy)) / (2 * hy)
        assert abs(gx - fx) <= 1e-6 * abs(gx) + 1e-9 * rc / x
        assert abs(gy - fy) <= 1e-6 * abs(gy) + 1e-9 * rc / y
