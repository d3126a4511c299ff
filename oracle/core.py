"""ctypes binding of the C oracle (lcdm_oracle.c).  Test infrastructure only."""
import ctypes
import numpy as np

from . import build as _build

OUT_NAMES = ("d_C", "t", "X", "d_M", "d_L", "mu")
C_KMS = 299792.458   # speed of light, km/s

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.oracle_quad_distances.argtypes = [dp, ctypes.c_int64, ctypes.c_int, ip, dp,
                                              ctypes.c_int64, ctypes.c_double, dp, dp]
        lib.oracle_carlson_distances.argtypes = [dp, ctypes.c_int64, ctypes.c_int, ip, dp,
                                                 ctypes.c_int64, dp, i32p, i32p, dp, dp]
        lib.oracle_quad_between.argtypes = [dp, ctypes.c_int64, ctypes.c_int, ip, dp, dp,
                                            ctypes.c_int64, ctypes.c_double, dp, dp]
        lib.oracle_quad_limits.argtypes = [dp, ctypes.c_int64, ctypes.c_int, dp, ctypes.c_double, dp, dp]
        lib.oracle_carlson_between.argtypes = [dp, ctypes.c_int64, ctypes.c_int, ip, dp, dp,
                                               ctypes.c_int64, dp, i32p, i32p, dp, dp]
        lib.oracle_carlson_limits.argtypes = [dp, ctypes.c_int64, ctypes.c_int, dp, dp, i32p, i32p, dp, dp]
        lib.oracle_carlson_batch.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp]
        lib.oracle_simpson.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_int64, dp]
        lib.oracle_set_mutation.argtypes = [ctypes.c_int]
        lib.oracle_legendre_distances.argtypes = [dp, ctypes.c_int64, ctypes.c_int, ip, dp, ctypes.c_int64, dp,
                                                  i32p, i32p, dp]
        lib.oracle_hyp2f1_flat.argtypes = [ctypes.c_double, ctypes.c_double, dp, ctypes.c_int64, dp]
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_mutation(m: int) -> None:
    """Plant a deliberate mistake (tests only); 0 restores the correct oracle."""
    _load().oracle_set_mutation(int(m))


_KIND = {"rf": 0, "rj": 1, "rc": 2, "rd": 3}


def carlson(kind: str, *args) -> np.ndarray:
    """Vectorised Carlson integral R_F / R_J / R_C / R_D (eqs. 2.6-2.9).

    Arguments broadcast; complex allowed.  Returns complex128.
    """
    arrs = np.broadcast_arrays(*[np.asarray(a, dtype=np.complex128) for a in args])
    shape = arrs[0].shape
    n = int(np.prod(shape)) if shape else 1
    packed = np.zeros((n, 8))
    for k, a in enumerate(arrs):
        a = a.reshape(-1)
        packed[:, 2 * k] = a.real
        packed[:, 2 * k + 1] = a.imag
    out = np.zeros((n, 2))
    _load().oracle_carlson_batch(_KIND[kind], n, _dp(packed), _dp(out))
    return (out[:, 0] + 1j * out[:, 1]).reshape(shape)


def _csr(params, z, offsets):
    params = np.ascontiguousarray(params, dtype=np.float64)
    if params.ndim == 1:
        params = params[None, :]
    z = np.ascontiguousarray(z, dtype=np.float64).reshape(-1)
    B, ncol = params.shape
    if offsets is None:
        if z.size % B:
            raise ValueError("dense layout needs nnz divisible by B")
        offsets = np.arange(B + 1, dtype=np.int64) * (z.size // B)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    return params, z, offsets, B, ncol


def quad_distances(params, z, offsets=None, rtol=1e-14, grad=False):
    """O1 (+ O4): quadrature of (2.3)-(2.5).  Returns out[nnz, 6] (OUT_NAMES)
    and, when grad, jac[nnz, 6, ncol] (derivatives w.r.t. the param columns)."""
    params, z, offsets, B, ncol = _csr(params, z, offsets)
    out = np.zeros((z.size, 6))
    jac = np.zeros((z.size, 6, ncol)) if grad else None
    _load().oracle_quad_distances(
        _dp(params), B, ncol, offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        _dp(z), z.size, rtol, _dp(out), _dp(jac) if grad else None)
    return (out, jac) if grad else out


def carlson_distances(params, z, offsets=None, roots=None, perm=None, return_imag=False):
    """O2: eqs. (3.7)-(3.9) / (B.1)-(B.3) from roots of E^2 in x = 1+z.

    roots/perm default to ``roots.roots_x`` / ``roots.permutations``.
    """
    from . import roots as _roots
    params, z, offsets, B, ncol = _csr(params, z, offsets)
    if roots is None:
        rho, nroot = _roots.roots_x(params)
    else:
        rho, nroot = roots
    if perm is None:
        perm = _roots.permutations(rho, nroot)
    packed = np.zeros((B, 4, 2))
    packed[:, :, 0] = rho.real
    packed[:, :, 1] = rho.imag
    packed = np.ascontiguousarray(packed)
    nroot = np.ascontiguousarray(nroot, dtype=np.int32)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    out = np.zeros((z.size, 6))
    imag = np.zeros((z.size, 3))
    i32p = ctypes.POINTER(ctypes.c_int32)
    _load().oracle_carlson_distances(
        _dp(params), B, ncol, offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        _dp(z), z.size, _dp(packed), nroot.ctypes.data_as(i32p), perm.ctypes.data_as(i32p),
        _dp(out), _dp(imag))
    return (out, imag) if return_imag else out


def dout_dz(params, z, offsets=None, rtol=1e-14):
    """Derivatives of O1's six outputs with respect to the redshift (the upper
    limit).  The derivative of each integral (2.3)-(2.5) with respect to its
    upper limit is its integrand there: (c/H0)/E, 1/(H0 (1+z) E),
    (c/H0)(1+z)^2/E, E from eq. (2.2); then d_M = (c/H0) S_k(D), D = chi H0/c,
    d_L = (1+z) d_M and mu (Sec. 2.1.1, fn22).  Returns [nnz, 6] in the order of
    OUT_NAMES; d mu/dz is 0 at z = 0 (mu = -inf there)."""
    params, z, offsets, B, ncol = _csr(params, z, offsets)
    o = quad_distances(params, z, offsets, rtol)
    rows = np.repeat(np.arange(B), np.diff(offsets))
    H0, Om, OL, Or = (params[rows, k] for k in range(4))
    Ok = params[rows, 4] if ncol == 5 else 1.0 - Om - OL - Or
    x = 1.0 + z
    E = np.sqrt(Or * x ** 4 + Om * x ** 3 + Ok * x ** 2 + OL)
    DH = C_KMS / H0
    tH = 977.7922216807891 / H0
    D, S = o[:, 0] / DH, o[:, 3] / DH
    r = np.sqrt(np.abs(Ok))
    SD = np.where(Ok > 0, np.cosh(r * D), np.where(Ok < 0, np.cos(r * D), 1.0))
    d = np.zeros((z.size, 6))
    d[:, 0] = DH / E
    d[:, 1] = tH / (x * E)
    d[:, 2] = DH * x * x / E
    d[:, 3] = DH * SD / E
    d[:, 4] = o[:, 3] + x * d[:, 3]
    with np.errstate(divide="ignore", invalid="ignore"):
        d[:, 5] = np.where(z > 0, 5.0 / np.log(10.0) * (1.0 / x + SD / (E * S)), 0.0)
    return d


def dmu_dz(params, z, offsets=None, rtol=1e-14):
    """d mu / d z of O1 (the last column of dout_dz):
    (5/ln 10) [1/(1+z) + S_k'(D) / (E S_k(D))]."""
    return dout_dz(params, z, offsets, rtol)[:, 5]


def _z1(z1, B):
    z1 = np.ascontiguousarray(np.broadcast_to(np.asarray(z1, dtype=np.float64), (B,)))
    return z1


def quad_between(params, z1, z2, offsets=None, rtol=1e-14, grad=False):
    """O1 (+ O4) with general limits: eqs. (2.3)-(2.5) from z1[b] (per row) to
    z2[j] (per pair).  Outputs as quad_distances; d_M is the transverse
    comoving distance S_k(chi(z1, z2)) and d_L = (1+z2) d_M / (1+z1)^2 (a
    source at z2 seen by a comoving observer at z1).  z2 < z1 gives NaN."""
    params, z2, offsets, B, ncol = _csr(params, z2, offsets)
    z1 = _z1(z1, B)
    out = np.zeros((z2.size, 6))
    jac = np.zeros((z2.size, 6, ncol)) if grad else None
    _load().oracle_quad_between(
        _dp(params), B, ncol, offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        _dp(z1), _dp(z2), z2.size, rtol, _dp(out), _dp(jac) if grad else None)
    return (out, jac) if grad else out


def quad_limits(params, z1, rtol=1e-14, grad=False):
    """O1 (+ O4) with the upper limit at infinity, per row: out[B, 2] =
    (chi(z1, inf) [Mpc], t(z1, inf) [Gyr]) -- the comoving distance to the
    particle horizon and the age of the universe at z1 (Sec. 2.1.1)."""
    params = np.ascontiguousarray(np.atleast_2d(params), dtype=np.float64)
    B, ncol = params.shape
    z1 = _z1(z1, B)
    out = np.zeros((B, 2))
    jac = np.zeros((B, 2, ncol)) if grad else None
    _load().oracle_quad_limits(_dp(params), B, ncol, _dp(z1), rtol, _dp(out),
                               _dp(jac) if grad else None)
    return (out, jac) if grad else out


def _roots_perm(params, roots, perm):
    from . import roots as _roots
    if roots is None:
        rho, nroot = _roots.roots_x(params)
    else:
        rho, nroot = roots
    if perm is None:
        perm = _roots.permutations(rho, nroot)
    B = params.shape[0]
    packed = np.zeros((B, 4, 2))
    packed[:, :, 0] = rho.real
    packed[:, :, 1] = rho.imag
    return (np.ascontiguousarray(packed), np.ascontiguousarray(nroot, dtype=np.int32),
            np.ascontiguousarray(perm, dtype=np.int32))


def carlson_between(params, z1, z2, offsets=None, roots=None, perm=None, return_imag=False):
    """O2 with general limits: eqs. (3.7)-(3.9) / (B.1)-(B.3) with
    X_m = sqrt(z2 - r_m), Y_m = sqrt(z1 - r_m) (Sec. 3.1); outputs as
    quad_between."""
    params, z2, offsets, B, ncol = _csr(params, z2, offsets)
    z1 = _z1(z1, B)
    packed, nroot, perm = _roots_perm(params, roots, perm)
    out = np.zeros((z2.size, 6))
    imag = np.zeros((z2.size, 3))
    i32p = ctypes.POINTER(ctypes.c_int32)
    _load().oracle_carlson_between(
        _dp(params), B, ncol, offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        _dp(z1), _dp(z2), z2.size, _dp(packed), nroot.ctypes.data_as(i32p), perm.ctypes.data_as(i32p),
        _dp(out), _dp(imag))
    return (out, imag) if return_imag else out


def carlson_limits(params, z1, roots=None, perm=None, return_imag=False):
    """O2 limits z2 -> infinity of eqs. (3.7)/(3.8) and (B.1)/(B.2), per row:
    out[B, 2] = (chi(z1, inf) [Mpc], t(z1, inf) [Gyr])."""
    params = np.ascontiguousarray(np.atleast_2d(params), dtype=np.float64)
    B, ncol = params.shape
    z1 = _z1(z1, B)
    packed, nroot, perm = _roots_perm(params, roots, perm)
    out = np.zeros((B, 2))
    imag = np.zeros((B, 2))
    i32p = ctypes.POINTER(ctypes.c_int32)
    _load().oracle_carlson_limits(_dp(params), B, ncol, _dp(z1), _dp(packed), nroot.ctypes.data_as(i32p),
                                  perm.ctypes.data_as(i32p), _dp(out), _dp(imag))
    return (out, imag) if return_imag else out


def simpson(param_row, z, n=1_000_000):
    """Brute-force composite Simpson rule of (2.3)-(2.5) on n subintervals."""
    p = np.ascontiguousarray(param_row, dtype=np.float64)
    res = np.zeros(3)
    _load().oracle_simpson(_dp(p), p.size, float(z), int(n), _dp(res))
    return res


def _legendre_raw(params, z, offsets, rho, nroot, ijkl):
    packed = np.zeros((params.shape[0], 4, 2))
    packed[:, :, 0] = np.nan_to_num(rho.real)
    packed[:, :, 1] = np.nan_to_num(rho.imag)
    out = np.zeros((z.size, 2))
    i32p = ctypes.POINTER(ctypes.c_int32)
    _load().oracle_legendre_distances(
        _dp(params), params.shape[0], params.shape[1], offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        _dp(z), z.size, _dp(np.ascontiguousarray(packed)), np.ascontiguousarray(nroot, dtype=np.int32).ctypes.data_as(i32p),
        np.ascontiguousarray(ijkl, dtype=np.int32).ctypes.data_as(i32p), _dp(out))
    return out


def legendre_assignment(params, zprobe=(0.5, 2.0, 8.0)):
    """Root assignment (i, j, k, l) of eqs. (B.4)-(B.7) per cosmology.  The
    formulas hold only for some orderings (App. B.2; the paper leaves the
    quartic choice open): the first permutation, in lexicographic order,
    whose comoving distance and time agree with the quadrature oracle to
    1e-8 at the probe redshifts is taken (-1 everywhere when none does)."""
    import itertools
    from . import roots as _roots
    params = np.ascontiguousarray(np.atleast_2d(params), dtype=np.float64)
    rho, nroot = _roots.roots_x(params)
    zp = np.asarray(zprobe, dtype=np.float64)
    res = np.full((params.shape[0], 4), -1, dtype=np.int32)
    for b in range(params.shape[0]):
        m = int(nroot[b])
        ref = quad_distances(params[b:b + 1], zp, np.array([0, zp.size]))
        for perm in itertools.permutations(range(m)):
            q = np.array(list(perm) + [0] * (4 - m), dtype=np.int32)
            with np.errstate(all="ignore"):
                got = _legendre_raw(params[b:b + 1], zp, np.array([0, zp.size], dtype=np.int64), rho[b:b + 1],
                                    nroot[b:b + 1], q[None, :])
            if np.all(np.isfinite(got)) and np.all(np.abs(got / ref[:, :2] - 1) < 1e-8):
                res[b] = q
                break
    return res, (rho, nroot)


def legendre_distances(params, z, offsets=None, assignment=None):
    """Eqs. (B.4)-(B.7): d_C [Mpc] and t [Gyr] in Legendre's form (App. B.2),
    F~ and Pi~ from Carlson's integrals (DLMF 19.25.5, 19.25.14), complex
    FP64.  Returns [nnz, 2] (NaN for rows without a valid assignment)."""
    params, z, offsets, B, ncol = _csr(params, z, offsets)
    if assignment is None:
        ijkl, (rho, nroot) = legendre_assignment(params)
    else:
        ijkl, (rho, nroot) = assignment
    out = _legendre_raw(params, z, offsets, rho, nroot, ijkl)
    rows = np.repeat(np.arange(B), np.diff(offsets))
    out[ijkl[rows, 0] < 0] = np.nan
    return out


def hyp2f1_flat_distance(H0, Om, z):
    """d_C [Mpc] of a flat radiationless cosmology by the hypergeometric
    solution (Sec. 3.2.2; x 2F1(1/2, 1/3; 4/3; -(Om/OL) x^3) / sqrt(OL))."""
    z = np.ascontiguousarray(z, dtype=np.float64).reshape(-1)
    out = np.zeros(z.size)
    _load().oracle_hyp2f1_flat(float(H0), float(Om), _dp(z), z.size, _dp(out))
    return out
