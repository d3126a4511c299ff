"""Operation count of the method per (cosmology, redshift) pair.

MEASUREMENT INFRASTRUCTURE ONLY (like the rest of ``oracle/``): used by
``bench.py`` to state the algorithmic work behind its roofline figure, and by
the tests that pin it.  Never part of the product path.

What is counted: the real single-precision operations of the Carlson
assembly of O2 -- eqs. (3.7)-(3.9) from the roots in complex arithmetic
(Sec. 3.1) -- for one pair at z1 = 0, and of its adjoint as the paper forms
it: reverse-mode differentiation through the assembly, with the Carlson
integrals as primitives whose gradients follow eqs. (2.10)-(2.12) (R_F: the
three R_D with each argument special; R_J: (2.11) and (2.12), the latter
with R_G, 6 R_G = sum_m x_m (x1 + x2 + x3 - x_m) R_D_m, in place of the
printed R_D; R_C = R_F(x, y, y) by (2.10)).  The duplication sequences
stop where Carlson's rule stops them at the 24-bit working precision
(r = 2^-24), so the counts are those of a single-precision evaluation; the
values themselves are carried in double precision (the unscaled complex
formulas of O2 overflow single precision for the big root ~ -Om/Or, which
is why the GPU path rescales them; the iteration counts do not depend on
that).

Conventions:
  * an operation is one real add/sub, mul, div, sqrt, or transcendental
    (log, exp, sin, cos, sinh, cosh); complex arithmetic is counted in the
    real operations it is made of (a complex product: 4 mul + 2 add);
  * per-cosmology work (roots, sqrt(-r_m), root differences d_ij, prefactors,
    the App. A root derivatives) is not counted: it is amortised over the
    row's pairs;
  * common subexpressions are evaluated once: the three u_ij, and one R_F for
    all outputs (the argument triples of (3.7), of (3.8) with i = A and of
    (3.9) with i = B are the same set, since u_ij = u_kl);
  * the adjoint carries a cotangent on each of d_C, t, X and mu and returns
    the derivatives with respect to the four roots (the per-cosmology App. A
    chain rule to the density parameters is not counted).
"""
import math

import numpy as np

COUNT = {"add": 0, "mul": 0, "div": 0, "sqrt": 0, "transc": 0}


def reset():
    for k in COUNT:
        COUNT[k] = 0


def snapshot():
    return dict(COUNT)


def _r(x):
    return float(x)


TAPE = []          # every node in creation order (a reverse topological order)
LAST_VALUES = None  # (chi, t, X) of the last pair_ops call, for the pins
LAST_RF_ITERS = 0   # duplication steps of the last rf call


class R:
    """A real with counted operations and a reverse-mode tape entry
    (parents with the local partial derivatives)."""
    __slots__ = ("v", "par", "g", "prim")

    def __init__(self, v, par=()):
        self.v = _r(v)
        self.par = par
        self.g = 0.0
        self.prim = None
        TAPE.append(self)

    def __add__(s, o):
        o = _lift(o)
        COUNT["add"] += 1
        return R(s.v + o.v, ((s, 1.0), (o, 1.0)))

    __radd__ = __add__

    def __sub__(s, o):
        o = _lift(o)
        COUNT["add"] += 1
        return R(s.v - o.v, ((s, 1.0), (o, -1.0)))

    def __rsub__(s, o):
        return _lift(o) - s

    def __neg__(s):
        return R(-s.v, ((s, -1.0),))

    def __mul__(s, o):
        o = _lift(o)
        COUNT["mul"] += 1
        return R(s.v * o.v, ((s, o.v), (o, s.v)))

    __rmul__ = __mul__

    def __truediv__(s, o):
        o = _lift(o)
        COUNT["div"] += 1
        q = s.v / o.v
        return R(q, ((s, 1.0 / o.v), (o, -q / o.v)))

    def __rtruediv__(s, o):
        return _lift(o) / s


def _lift(x):
    return x if isinstance(x, R) else R(x)


def _defer_to_complex(f):
    """Real-by-complex operations are the complex type's (its reflected method)."""
    def g(s, o):
        if isinstance(o, C):
            return NotImplemented
        return f(s, o)
    return g


for _name in ("__add__", "__radd__", "__sub__", "__rsub__", "__mul__", "__rmul__", "__truediv__", "__rtruediv__"):
    setattr(R, _name, _defer_to_complex(getattr(R, _name)))


def rsqrt_(x):
    COUNT["sqrt"] += 1
    v = math.sqrt(x.v) if x.v > 0 else 0.0
    return R(v, ((x, 0.5 / v if v > 0 else 0.0),))


def transc(f, df, x):
    COUNT["transc"] += 1
    return R(f(x.v), ((x, df(x.v)),))


class C:
    """A complex number of two counted reals."""
    __slots__ = ("re", "im")

    def __init__(self, re, im=0.0):
        self.re = _lift(re)
        self.im = _lift(im)

    def __add__(s, o):
        o = _clift(o)
        return C(s.re + o.re, s.im + o.im)

    __radd__ = __add__

    def __sub__(s, o):
        o = _clift(o)
        return C(s.re - o.re, s.im - o.im)

    def __rsub__(s, o):
        return _clift(o) - s

    def __neg__(s):
        return C(-s.re, -s.im)

    def __mul__(s, o):
        if isinstance(o, (R, float, int)):
            o = _lift(o)
            return C(s.re * o, s.im * o)
        return C(s.re * o.re - s.im * o.im, s.re * o.im + s.im * o.re)

    __rmul__ = __mul__

    def __truediv__(s, o):
        if isinstance(o, (R, float, int)):
            inv = 1.0 / _lift(o)
            return C(s.re * inv, s.im * inv)
        den = o.re * o.re + o.im * o.im
        inv = 1.0 / den
        return C((s.re * o.re + s.im * o.im) * inv, (s.im * o.re - s.re * o.im) * inv)

    def __rtruediv__(s, o):
        return _clift(o) / s


def _clift(x):
    return x if isinstance(x, C) else C(x)


def cabs(z):
    return rsqrt_(z.re * z.re + z.im * z.im)


def csqrt(z):
    """Principal square root."""
    r = cabs(z)
    if z.re.v >= 0:
        t = rsqrt_((r + z.re) * 0.5)
        return C(t, z.im / (t + t)) if t.v > 0 else C(t, 0.0)
    t = rsqrt_((r - z.re) * 0.5)
    a = z.im if z.im.v >= 0 else -z.im
    re = a / (t + t)
    return C(re, t if z.im.v >= 0 else -t)


def _detach(z):
    """Value copy without tape links (the Carlson primitives are not taped)."""
    return C(R(z.re.v), R(z.im.v))


# ---------------------------------------------------------------------------
# Carlson integrals by duplication (ref. [10] of the paper) at r = 2^-24.
# ---------------------------------------------------------------------------
_RTOL = 2.0 ** -24


def _maxabs(*zs):
    return max(cabs(z).v for z in zs)


def rf(x, y, z):
    x0, y0 = x, y
    A0 = (x + y + z) * (1.0 / 3.0)
    A = A0
    Q = (3 * _RTOL) ** (-1 / 6) * _maxabs(A0 - x, A0 - y, A0 - z)
    f = 1.0
    global LAST_RF_ITERS
    LAST_RF_ITERS = 0
    while f * Q >= cabs(A).v:
        sx, sy, sz = csqrt(x), csqrt(y), csqrt(z)
        lam = sx * sy + sx * sz + sy * sz
        A, x, y, z = (A + lam) * 0.25, (x + lam) * 0.25, (y + lam) * 0.25, (z + lam) * 0.25
        f *= 0.25
        LAST_RF_ITERS += 1
    X = (A0 - x0) * f / A
    Y = (A0 - y0) * f / A
    Z = -(X + Y)
    E2 = X * Y - Z * Z
    E3 = X * Y * Z
    s = 1.0 - E2 * 0.1 + E3 * (1 / 14) + E2 * E2 * (1 / 24) - E2 * E3 * (3 / 44)
    return s / csqrt(A)


def rc(x, y):
    A0 = (x + y * 2.0) * (1.0 / 3.0)
    A = A0
    Q = (3 * _RTOL) ** (-1 / 8) * cabs(A0 - x).v
    f = 1.0
    while f * Q >= cabs(A).v:
        lam = csqrt(x) * csqrt(y) * 2.0 + y
        A, x, y = (A + lam) * 0.25, (x + lam) * 0.25, (y + lam) * 0.25
        f *= 0.25
    s = (y - A) / A
    ser = 1.0 + s * s * (0.3 + s * (1 / 7 + s * (3 / 8 + s * (9 / 22 + s * (159 / 208 + s * (9 / 8))))))
    return ser / csqrt(A)


def rj(x, y, z, p):
    x0, y0, z0 = x, y, z
    A0 = (x + y + z + p * 2.0) * 0.2
    A = A0
    delta = (p - x) * (p - y) * (p - z)
    Q = (_RTOL / 4) ** (-1 / 6) * max(_maxabs(A0 - x, A0 - y, A0 - z), cabs(A0 - p).v)
    f = 1.0
    acc = C(0.0)
    while f * Q >= cabs(A).v:
        sx, sy, sz, sp = csqrt(x), csqrt(y), csqrt(z), csqrt(p)
        lam = sx * sy + sx * sz + sy * sz
        d = (sp + sx) * (sp + sy) * (sp + sz)
        e = delta * (f * f * f) / (d * d)
        acc = acc + rc(C(1.0), e + 1.0) * f / d
        A, x, y, z, p = (A + lam) * 0.25, (x + lam) * 0.25, (y + lam) * 0.25, (z + lam) * 0.25, (p + lam) * 0.25
        f *= 0.25
    X = (A0 - x0) * f / A
    Y = (A0 - y0) * f / A
    Z = (A0 - z0) * f / A
    P = -(X + Y + Z) * 0.5
    E2 = X * Y + X * Z + Y * Z - P * P * 3.0
    E3 = X * Y * Z + E2 * P * 2.0 + P * P * P * 4.0
    E4 = (X * Y * Z * 2.0 + E2 * P + P * P * P * 3.0) * P
    E5 = X * Y * Z * P * P
    s = (1.0 - E2 * (3 / 14) + E3 * (1 / 6) + E2 * E2 * (9 / 88) - E4 * (3 / 22) - E2 * E3 * (9 / 52)
         + E5 * (3 / 26))
    return s * f / (A * csqrt(A)) + acc * 6.0


def rd(x, y, z):
    return rj(x, y, z, z)


def rj_pv(x, y, z, p):
    """R_J with the principal value for negative real p (Sec. 2.2); z real."""
    if p.im.v != 0 or p.re.v >= 0:
        return rj(x, y, z, p)
    q = -p
    s = (z * (x + y + q) - x * y) / (z + q)
    xy = x * y
    return ((s - z) * rj(x, y, z, s) - rf(x, y, z) * 3.0
            + csqrt(xy * z / (xy + s * q)) * rc_pv(xy + s * q, s * q) * 3.0) / (q + z)


def rc_pv(x, y):
    if y.im.v == 0 and y.re.v < 0:
        q = -y
        return csqrt(x / (x + q)) * rc(x + q, q)
    return rc(x, y)


# ---------------------------------------------------------------------------
# Primitives with gradient rules (2.10)-(2.12): value, and a function that
# maps the value's cotangent to the arguments' cotangents (counted).
# ---------------------------------------------------------------------------
class Prim:
    """Shared R_D values of one argument triple (computed on first use)."""

    def __init__(self, x):
        self.x = [_detach(v) for v in x]
        self._rd = None

    def rds(self):
        if self._rd is None:
            a, b, c = self.x
            self._rd = [rd(b, c, a), rd(c, a, b), rd(a, b, c)]   # R_D with x_m special
        return self._rd


def rf_prim(pr):
    v = rf(*pr.x)

    def back(g):
        return [g * (D * (-1.0 / 6.0)) for D in pr.rds()]       # eq. (2.10)
    return v, back


def rj_prim(pr, p):
    p = _detach(p)
    J = rj_pv(*pr.x, p)

    def back(g):
        x = pr.x
        D = pr.rds()
        dx = [(J - D[m]) / ((p - x[m]) * 2.0) for m in range(3)]                   # eq. (2.11)
        e1 = x[0] + x[1] + x[2]
        RG = sum(((x[m] * (e1 - x[m]) * D[m]) for m in range(3)), C(0.0)) * (1 / 6)
        F = rf(*x)
        prod = (p - x[0]) * (p - x[1]) * (p - x[2])
        sq = csqrt(x[0] * x[1] * x[2])
        inv = sum((1.0 / (p - x[m]) for m in range(3)), C(0.0))
        dp = ((p * p * F - p * RG * 2.0 + sq) / (p * prod) - inv * J * (1 / 3)) * 1.5   # eq. (2.12), R_G
        return [g * d for d in dx] + [g * dp]
    return J, back


def rd_prim(pr, m):
    """R_D with the m-th argument special, from the shared values; its
    gradient: dR_D(x,y,z)/dx = (R_D(x,y,z) - R_D(y,z,x)) / (2 (z - x)) for the
    other two arguments and homogeneity (degree -3/2) for the special one."""
    D = pr.rds()
    v = D[m]

    def back(g):
        x = pr.x
        o = [q for q in range(3) if q != m]
        d = [(v - D[q]) / ((x[m] - x[q]) * 2.0) for q in o]
        dm = (v * (-1.5) - x[o[0]] * d[0] - x[o[1]] * d[1]) / x[m]
        out = [None, None, None]
        out[o[0]], out[o[1]], out[m] = g * d[0], g * d[1], g * dm
        return out
    return v, back


def rc_prim(x, y):
    x, y = _detach(x), _detach(y)
    v = rc_pv(x, y)

    def back(g):
        # R_C(x, y) = R_F(x, y, y): eq. (2.10)
        return [g * (rd(y, y, x) * (-1.0 / 6.0)), g * (rd(x, y, y) * (-2.0 / 6.0))]
    return v, back


# ---------------------------------------------------------------------------
# One pair: forward (3.7)-(3.9), observables, and the adjoint.
# ---------------------------------------------------------------------------
def _taped_complex(v):
    return C(R(v.real), R(v.imag))


def pair_ops(rho, iX, lX, it, H0, Ok, z, grad=True, cot=("d_C", "t", "X", "mu")):
    """Counted operations for one pair (quartic reduction) at redshift z.
    rho: the four roots of E^2 in x = 1 + z (complex); it, iX, lX the root
    labels of (3.8) and (3.9); cot: the outputs that carry a cotangent in the
    adjoint.  Returns the operation counts of the forward pass (all four
    outputs) and of the adjoint."""
    reset()
    TAPE.clear()
    r = [complex(v) - 1.0 for v in rho]                  # roots in z
    rr = [_taped_complex(v) for v in r]                  # taped leaves (cotangents wanted)
    Y = [C(math.sqrt(-v.real) if v.imag == 0 else complex(np.sqrt(-v)).real,
           0.0 if v.imag == 0 else complex(np.sqrt(-v)).imag) for v in r]   # per cosmology
    zc = R(z)
    X = [csqrt(zc - rr[m]) for m in range(4)]            # per pair

    def uab(a, b):
        c, d = [m for m in range(4) if m not in (a, b)]
        return X[a] * X[b] * Y[c] * Y[d] + Y[a] * Y[b] * X[c] * X[d]

    u01, u02, u03 = uab(0, 1), uab(0, 2), uab(0, 3)
    U = {frozenset((0, 1)): u01, frozenset((2, 3)): u01, frozenset((0, 2)): u02, frozenset((1, 3)): u02,
         frozenset((0, 3)): u03, frozenset((1, 2)): u03}
    sq = [u01 * u01, u02 * u02, u03 * u03]
    prim = Prim(sq)
    RF, RFb = rf_prim(prim)

    def use(vals, inputs, back):
        ph = C(R(vals.re.v), R(vals.im.v))
        ph.re.prim = (back, inputs, ph)
        return ph

    RFv = use(RF, sq, RFb)
    dz = zc
    chi = RFv * dz * 2.0
    # t, eq. (3.8), i = it
    i = it
    j, k, l = [m for m in range(4) if m != i]
    dij, dik, dil = rr[j] - rr[i], rr[k] - rr[i], rr[l] - rr[i]
    di5, dj5, dk5, dl5 = [-(rr[m] + 1.0) for m in (i, j, k, l)]
    uij = U[frozenset((i, j))]
    ui5 = uij * uij - dz * dz * dik * dil * dj5 / di5
    qi5 = (zc + 1.0) / (zc - rr[i]) / (-rr[i]) * ui5
    si5 = qi5 + dz * dz * dk5 * dl5 * dj5 / di5
    J5, J5b = rj_prim(prim, ui5)
    J5v = use(J5, sq + [ui5], J5b)
    RC5, RC5b = rc_prim(si5, qi5)
    RC5v = use(RC5, [si5, qi5], RC5b)
    t = dz * 2.0 / (rr[i] + 1.0) * (RFv - (dz * dz * (1 / 3) * dij * dik * dil / di5 * J5v + RC5v))
    # X, eq. (3.9), i = iX, l = lX
    i, l = iX, lX
    j, k = [m for m in range(4) if m not in (i, l)]
    dij, dik, dil = rr[j] - rr[i], rr[k] - rr[i], rr[l] - rr[i]
    djl, dkl = rr[l] - rr[j], rr[l] - rr[k]
    uil = U[frozenset((i, l))]
    ui0 = U[frozenset((i, j))] * U[frozenset((i, j))] - dz * dz * dik * dil
    qi0 = ui0 / (zc - rr[i]) / (-rr[i])
    si0 = qi0 + dz * dz
    Jx, Jxb = rj_prim(prim, ui0)
    Jxv = use(Jx, sq + [ui0], Jxb)
    RCx, RCxb = rc_prim(si0, qi0)
    RCxv = use(RCx, [si0, qi0], RCxb)
    # R_D with the argument u_il^2 special: one of the shared R_D values
    RDl, RDlb = rd_prim(prim, [u01, u02, u03].index(U[frozenset((i, l))]))
    RDv = use(RDl, sq, RDlb)
    sumr = rr[0] + rr[1] + rr[2] + rr[3] + 4.0
    term0 = (X[i] * X[j] * X[k] / X[l] - Y[i] * Y[j] * Y[k] / Y[l]) / dz
    term1 = ((rr[i] + 1.0) * (rr[i] + 1.0) * 2.0 - dij * dik) * RFv
    term2 = djl * dkl * (dz * dz * (1 / 3) * dij * dik * RDv + X[i] * Y[i] / (X[l] * Y[l]) / uil)
    term3 = sumr * (dz * dz * (1 / 3) * dij * dik * dil * (-1.0) * Jxv + RCxv)
    Xd = dz * (term0 + term1 + term2 + term3)
    # observables: curvature map (sinh / sin), d_M, d_L, mu
    D = chi.re * (1.0 / 1.0)
    sk = math.sqrt(abs(Ok)) if Ok != 0 else 1.0
    arg = D * sk
    S = transc(math.sinh if Ok > 0 else math.sin, math.cosh if Ok > 0 else math.cos, arg) / sk
    dL = S * (zc + 1.0)
    mu = transc(math.log, lambda v: 1.0 / v, dL) * (5.0 / math.log(10.0)) + 25.0
    fwd = snapshot()
    global LAST_VALUES
    LAST_VALUES = (chi.re.v, t.re.v, Xd.re.v)          # in units of Or^-1/2 c/H0, Or^-1/2/H0, Or^-1/2 c/H0
    if not grad:
        TAPE.clear()
        return fwd, None
    reset()
    # one reverse sweep in reverse creation order: cotangent 1 on d_C, t, X and
    # mu (the real parts); each tape edge is one multiply-add, each Carlson
    # primitive maps its value's cotangent to its arguments by its rule
    for name, o in (("d_C", chi.re), ("t", t.re), ("X", Xd.re), ("mu", mu)):
        if name in cot:
            o.g = 1.0
    nodes = list(TAPE)
    for v in reversed(nodes):
        if v.prim is not None and (v.g != 0.0 or v.prim[2].im.g != 0.0):
            back, inputs, ph = v.prim
            gs = back(C(R(ph.re.g), R(ph.im.g)))
            for inp, gi in zip(inputs, gs):
                COUNT["add"] += 2
                inp.re.g += gi.re.v
                inp.im.g += gi.im.v
            continue
        if v.g == 0.0:
            continue
        for p, d in v.par:
            COUNT["mul"] += 1
            COUNT["add"] += 1
            p.g += v.g * d
    adj = snapshot()
    TAPE.clear()
    return fwd, adj


def batch_counts(params, z, offsets, nsample=400, seed=0, cot=("d_C", "t", "X", "mu")):
    """Mean counts per pair over a random sample of a batch (quartic rows),
    with the oracle's roots and root labels."""
    from . import roots as _roots
    params = np.atleast_2d(np.asarray(params, dtype=np.float64))
    rho, nroot = _roots.roots_x(params)
    perm = _roots.permutations(rho, nroot)
    rng = np.random.default_rng(seed)
    idx = rng.choice(z.size, min(nsample, z.size), replace=False)
    rows = np.searchsorted(offsets, idx, side="right") - 1
    tot_f = {k: 0 for k in COUNT}
    tot_a = {k: 0 for k in COUNT}
    n = 0
    for p, row in zip(idx, rows):
        if nroot[row] != 4 or z[p] <= 0:
            continue
        ncol = params.shape[1]
        Om, OL, Or = params[row, 1:4]
        Ok = params[row, 4] if ncol >= 5 else 1.0 - Om - OL - Or
        f, a = pair_ops(rho[row], perm[row, 1], perm[row, 2], perm[row, 0], params[row, 0], Ok, float(z[p]),
                        cot=cot)
        for k in COUNT:
            tot_f[k] += f[k]
            tot_a[k] += a[k]
        n += 1
    return {"pairs": n, "forward": {k: v / n for k, v in tot_f.items()},
            "adjoint": {k: v / n for k, v in tot_a.items()}}


if __name__ == "__main__":
    # The count behind the benchmark's algorithmic roofline: a random sample
    # of the general batch (4096 cosmologies x 1024 redshifts, seed 2), with
    # the redshifts rounded to float32 as the benchmark feeds them; forward
    # d_C, t, X, mu and the adjoint of the cotangents the benchmark step
    # carries (d_C, t, mu).
    import json
    import sys
    sys.path.insert(0, __import__("os").path.dirname(__import__("os").path.dirname(__import__("os").path.abspath(__file__))))
    from paper_2212_01937_gb300 import workloads
    nsample = int(sys.argv[1]) if len(sys.argv) > 1 else 1000
    b = workloads.general_batch()
    res = batch_counts(b.params, b.z.astype(np.float32).astype(np.float64), b.offsets, nsample=nsample, seed=0,
                       cot=("d_C", "t", "mu"))
    tot = {k: res["forward"][k] + res["adjoint"][k] for k in COUNT}
    res["total"] = tot
    res["flops_per_pair"] = tot["add"] + tot["mul"]
    res["mufu_per_pair"] = tot["div"] + tot["sqrt"] + tot["transc"]
    print(json.dumps(res, indent=1))
