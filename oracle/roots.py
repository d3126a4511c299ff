"""O3: roots of E^2 and their derivatives (test infrastructure only).

* Factorisation (3.2): E^2(x) = alpha_m prod_j (x - rho_j) with x = 1 + z, so
  the roots in z are r_j = rho_j - 1.  Roots are the eigenvalues of the
  companion matrix (the numerical route of Sec. 3, fn12), then polished by
  Newton steps on the original polynomial with an exact (rational) residual.
* App. A, eqs. (A.1)-(A.4): the derivatives of the roots with respect to the
  monic coefficients c_k solve  1 = C^T (dr/dc),  where row j of C holds the
  coefficients of prod_{i != j} (x - rho_i) (Vieta's formulae); here the
  linear system is solved as written, with numpy.
"""
import numpy as np


def poly_coeffs_x(params):
    """Coefficients of E^2 in x = 1+z, lowest power first (eq. 2.2):
    [OL, Ox, Ok + Os, Om, Or].  params rows (H0, Om, OL, Or[, Ok[, Os, Ox]]);
    closure Ok = 1 - Om - OL - Or when only four columns are given (Sec. 2.1);
    Os (w = -1/3) and Ox (w = -2/3) are the further components of fn4, zero
    unless given."""
    p = np.atleast_2d(np.asarray(params, dtype=np.float64))
    Om, OL, Or = p[:, 1], p[:, 2], p[:, 3]
    Ok = p[:, 4] if p.shape[1] >= 5 else 1.0 - Om - OL - Or
    Os = p[:, 5] if p.shape[1] >= 7 else np.zeros_like(OL)
    Ox = p[:, 6] if p.shape[1] >= 7 else np.zeros_like(OL)
    return np.stack([OL, Ox, Ok + Os, Om, Or], axis=1)


def _polish(coef_low, x, iters=6):
    """Newton's method on sum_k coef_low[k] x^k for each root x (complex),
    with the residual p(x) and p'(x) evaluated exactly in rational arithmetic
    (the float coefficients and the float iterate are exact rationals), so the
    only rounding is that of the new iterate to double.  Near a double root
    (the no-Big-Bang boundary, Fig. 1) a double-precision residual is all
    rounding noise once |p'| is small; the exact one still converges to the
    root of the stated polynomial, to within the rounding of its parts."""
    from fractions import Fraction as F
    c = [F(float(a)) for a in coef_low]
    out = np.array(x, dtype=np.complex128)
    for j in range(out.size):
        xr, xi = F(float(out[j].real)), F(float(out[j].imag))
        for _ in range(iters):
            pr, pi, dr, di = c[-1], F(0), F(0), F(0)
            for a in c[-2::-1]:                      # Horner, highest power first
                dr, di = dr * xr - di * xi + pr, dr * xi + di * xr + pi
                pr, pi = pr * xr - pi * xi + a, pr * xi + pi * xr
            den = dr * dr + di * di
            if den == 0:
                break
            sr = (pr * dr + pi * di) / den               # p / p'
            si = (pi * dr - pr * di) / den
            nr, ni = F(float(xr - sr)), F(float(xi - si))
            if nr == xr and ni == xi:
                break
            xr, xi = nr, ni
        out[j] = complex(float(xr), float(xi))
    return out


def roots_x(params, real_tol=1e-10):
    """Roots rho of E^2 in x for each cosmology.

    Returns (rho[B, 4] complex, nroot[B]) with nroot = 4 (Or > 0, quartic) or
    3 (Or == 0, cubic; rho[:, 3] = nan).  Roots whose imaginary part is below
    real_tol relative to their modulus are made exactly real, and a complex
    pair is made exactly conjugate (E^2 has real coefficients, Sec. 3)."""
    coef = poly_coeffs_x(params)
    B = coef.shape[0]
    rho = np.full((B, 4), np.nan + 0j)
    nroot = np.zeros(B, dtype=np.int32)
    for b in range(B):
        c = coef[b]
        deg = 4 if c[4] != 0 else 3
        lead = c[deg]
        mon = c[:deg] / lead                       # monic c_0..c_{deg-1}
        comp = np.zeros((deg, deg))
        comp[1:, :-1] = np.eye(deg - 1)
        comp[:, -1] = -mon
        x = np.linalg.eigvals(comp).astype(np.complex128)
        x = _polish(c[:deg + 1], x)
        isreal = np.abs(x.imag) <= real_tol * np.abs(x)
        x = np.where(isreal, x.real + 0j, x)
        # exact conjugacy for the complex ones
        cx = np.where(~isreal)[0]
        if cx.size == 2:
            a = 0.5 * (x[cx[0]] + np.conj(x[cx[1]]))
            x[cx[0]], x[cx[1]] = a, np.conj(a)
        elif cx.size == 4:
            used = []
            for i in cx:
                if i in used:
                    continue
                j = min((k for k in cx if k != i and k not in used),
                        key=lambda k: abs(x[k] - np.conj(x[i])))
                a = 0.5 * (x[i] + np.conj(x[j]))
                x[i], x[j] = a, np.conj(a)
                used += [i, j]
        rho[b, :deg] = x
        nroot[b] = deg
    return rho, nroot


def classify_roots(rho, nroot):
    """Per cosmology: (n_real, no_big_bang).  No Big Bang (Sec. 3, Fig. 1):
    a real root of E^2 at z >= 0, i.e. rho >= 1, lies on the integration path."""
    B = rho.shape[0]
    nreal = np.zeros(B, dtype=np.int32)
    nobb = np.zeros(B, dtype=bool)
    for b in range(B):
        x = rho[b, :nroot[b]]
        re = x.imag == 0
        nreal[b] = re.sum()
        nobb[b] = bool(np.any(re & (x.real >= 1.0)))
    return nreal, nobb


def permutations(rho, nroot):
    """Root labels used by O2, per cosmology: (i_t, i_X, l_X).

    * t, eq. (3.8): i = root of E^2(z+1) with the largest modulus (fn15).
    * X, eq. (3.9): l = that same root, i = the real root with the next
      largest modulus (the ordering found best for (3.9) in double precision).
    * Cubic (B.2)/(B.3): i = the real root of largest modulus (i_t = i_X).
    """
    B = rho.shape[0]
    perm = np.zeros((B, 3), dtype=np.int32)
    for b in range(B):
        m = nroot[b]
        x = rho[b, :m]
        order = np.argsort(-np.abs(x), kind="stable")
        reals = [k for k in order if x[k].imag == 0]
        if m == 4:
            it = order[0]
            lX = order[0]
            cand = [k for k in reals if k != lX]
            iX = cand[0] if cand else order[1]
            perm[b] = (it, iX, lX)
        else:
            i = reals[0] if reals else order[0]
            perm[b] = (i, i, i)
    return perm


def root_coef_jacobian(rho):
    """App. A: D[i, j] = d rho_j / d c_i for the monic polynomial with roots
    rho (length m), by solving (A.3)-(A.4) as a linear system.

    (A.3) at each power z^k: delta_ik = -sum_j D[i, j] C[j, k], with C[j, :]
    the coefficients (lowest first) of prod_{n != j} (z - rho_n)."""
    rho = np.asarray(rho, dtype=np.complex128)
    m = rho.size
    C = np.zeros((m, m), dtype=np.complex128)
    for j in range(m):
        others = np.delete(rho, j)
        C[j] = np.poly(others)[::-1]             # lowest power first, length m
    # I = -D C  ->  D = -C^{-1}, computed as a solve of C^T D^T = -I
    D = np.linalg.solve(C.T, -np.eye(m)).T
    return D


def root_param_jacobian(params, rho, nroot):
    """d rho_j / d theta for theta = the Omega columns of params (Om, OL, Or[, Ok]),
    via the App. A coefficient Jacobian and c_k = alpha_k / alpha_m.

    Returns jac[B, 4, ncol-1] complex (nan where undefined, e.g. Or for a
    cubic)."""
    p = np.atleast_2d(np.asarray(params, dtype=np.float64))
    B, ncol = p.shape
    coef = poly_coeffs_x(p)                     # alpha_0..alpha_4
    out = np.full((B, 4, ncol - 1), np.nan + 0j)
    for b in range(B):
        m = nroot[b]
        D = root_coef_jacobian(rho[b, :m])       # [i (coef), j (root)]
        alpha = coef[b]
        am = alpha[m]
        # d alpha_k / d theta: alpha = (OL, 0, Ok, Om, Or); closure couples Ok.
        dalpha = np.zeros((5, ncol - 1))
        for ip in range(ncol - 1):               # 0:Om 1:OL 2:Or 3:Ok
            if ip == 0: dalpha[3, ip] = 1
            if ip == 1: dalpha[0, ip] = 1
            if ip == 2: dalpha[4, ip] = 1
            if ip == 3: dalpha[2, ip] = 1
            if ncol == 4 and ip < 3:
                dalpha[2, ip] = -1               # Ok = 1 - Om - OL - Or
        for ip in range(ncol - 1):
            if m == 3 and ip == 2:
                continue                         # no Or direction for a cubic
            # c_k = alpha_k / alpha_m, k < m
            dc = (dalpha[:m, ip] * am - alpha[:m] * dalpha[m, ip]) / am ** 2
            out[b, :m, ip] = dc @ D
    return out
