// Distance assembly for one (cosmology, redshift) pair, written once for any
// scalar S: a plain number (values only) or Dual<T,K> (values and tangents
// with respect to the density parameters).
//
// Carlson integrals enter through carlson_any / rc_any.  Their tangents are
// carried through one shared duplication sequence as dual numbers (see
// carlson_any); R_C's tangents use dR_F/dx_m = -R_D(..x_m..)/6 (eq. 2.10) with
// R_C(x, y) = R_F(x, y, y) and Euler's relation for the R_D that has a pair
// member special (rc_value_grad).  All R_D, R_J and R_F values of a pair come
// from one shared duplication sequence.
//
// Cauchy principal values (Sec. 2.2) for negative p or y:
//   (q+z) R_J(x,y,z,-q) = (s-z) R_J(x,y,z,s) - 3 R_F + 3 sqrt(xyz/(xy+sq)) R_C(xy+sq, sq),
//   s = (z(x+y+q) - xy)/(z+q), z the real member of the triple;
//   R_C(x, -q) = sqrt(x/(x+q)) R_C(x+q, q).
#pragma once
#include "lcdm_math.cuh"

namespace lcdm {


// ---------------------------------------------------------------- values ----
template <class T> LCDM_HD T rc_any(T x, T y, int* fail) {
    if (sval(y) < 0) {
        T x2 = x - y, y2 = -y;
        return ssqrt(x / x2) * rc_value(x2, y2, fail);
    }
    return rc_value(x, y, fail);
}

// The triple enters through square roots: x1 = u1^2 and the pair y = u^2
// (a conjugate pair, or two reals).  The R_J tracks are given by
// h_j = p_j - x1 (their distance from the single argument): the callers form
// h_j directly, without cancellation.  NEED_RD1: return R_D(y_a, y_b, x1);
// WANT_DJ: return DJ = (R_J(last track) - R_D1) / h.  Written once for plain
// and dual numbers: tangents are carried through the duplication sequence
// itself (see carlson_sym; the note below on why not by (2.10)-(2.12)).
template <int NJ, bool NEED_RD1, bool WANT_DJ, class T, class PT>
LCDM_HD void carlson_any(const T& u1, const PT& up, const T* h, T& RF, T& RD1, T* RJ, int* fail, T* DJ = 0) {
    const T x1 = u1 * u1;
    const PT pr = up * up;
    T tr[NJ > 0 ? NJ : 1], s[NJ > 0 ? NJ : 1], q[NJ > 0 ? NJ : 1], hh[NJ > 0 ? NJ : 1], dl[NJ > 0 ? NJ : 1];
    bool pv[NJ > 0 ? NJ : 1];
#pragma unroll
    for (int j = 0; j < NJ; j++) {
        T p = x1 + h[j];
        pv[j] = sval(vof(p)) < 0;
        if (pv[j]) {
            q[j] = -p;
            s[j] = (x1 * (psum(pr) + q[j]) - pprod(pr)) / (x1 + q[j]);
            if (!(sval(vof(s[j])) > 0)) *fail = 2;
            tr[j] = s[j];
            hh[j] = s[j] - x1;
        } else {
            tr[j] = p;
            hh[j] = h[j];
        }
        // (p - x1)(p - y_a)(p - y_b) from the members: |p - y|^2 has no cancellation
        dl[j] = hh[j] * pprod(prsub(tr[j], pr));
    }
    constexpr int JL = NJ > 0 ? NJ - 1 : 0;
    const T PiL = WANT_DJ ? pprod(prsub(tr[JL], pr)) : x1;
    SymResult<T, NJ> R = carlson_sym<T, NJ, NEED_RD1 || WANT_DJ, WANT_DJ>(
        sabs(u1), proot_sum(up), proot_prod(up), pis_cplx(up), tr, dl, fail, hh[JL], PiL);
    RF = R.RF;
    RD1 = R.RD1;
    // principal values (the tracks ran at s_j)
#pragma unroll
    for (int j = 0; j < NJ; j++) {
        if (!pv[j]) {
            RJ[j] = R.RJ[j];
        } else {
            T xy = pprod(pr), sq = s[j] * q[j];
            T rc = rc_any(xy + sq, sq, fail);
            RJ[j] = ((s[j] - x1) * R.RJ[j] - RF * cst<typename Base<T>::type>(3.0)
                     + ssqrt(x1 * xy / (xy + sq)) * rc * cst<typename Base<T>::type>(3.0)) / (q[j] + x1);
        }
    }
    if constexpr (WANT_DJ && NJ > 0) {
        *DJ = R.DJ;
        if (pv[JL]) *DJ = (RJ[JL] - RD1) / h[JL];
    }
}

// --------------------------------------------------------------- tangents ---
// R_C(x, y) = R_F(x, y, y) (eq. 2.8) and its two partial derivatives from one
// symmetric duplication sequence with the pair (y, y): dR_C/dx = -R_D(y, y, x)/6
// (eq. 2.10) and dR_C/dy = -2 R_D(x, y, y)/6, where R_D(x, y, y) follows from
// Euler's relation for R_F (homogeneous of degree -1/2),
//   x R_D(y, y, x) + 2 y R_D(x, y, y) = 3 R_C,
// a difference whose terms are within a factor 20 of it for x/y in [1e-8, 1e8].
template <class T> struct RcGrad { T v, gx, gy; };
template <class T> LCDM_NI RcGrad<T> rc_value_grad(T x, T y, int* fail) {
    const T sy = ssqrt(y);
    SymResult<T, 0> R = carlson_sym<T, 0, true>(ssqrt(x), sy + sy, y, false, (const T*)0, (const T*)0, fail);
    RcGrad<T> g;
    g.v = R.RF;
    g.gx = R.RD1 * cst<T>(-1.0 / 6.0);
    g.gy = (x * R.RD1 - cst<T>(3.0) * R.RF) / (cst<T>(6.0) * y);
    return g;
}
template <class T, int K> LCDM_HD Dual<T, K> rc_dual_pos(const Dual<T, K>& x, const Dual<T, K>& y, int* fail) {
    const RcGrad<T> g = rc_value_grad<T>(x.v, y.v, fail);
    Dual<T, K> r;
    r.v = g.v;
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = g.gx * x.d[k] + g.gy * y.d[k];
    return r;
}
template <class T, int K> LCDM_HD Dual<T, K> rc_any(const Dual<T, K>& x, const Dual<T, K>& y, int* fail) {
    if (sval(y.v) < 0) {
        Dual<T, K> x2 = x - y, y2 = -y;
        return ssqrt(x / x2) * rc_dual_pos(x2, y2, fail);
    }
    return rc_dual_pos(x, y, fail);
}

// Tangents of R_F, R_D and R_J are carried through the duplication sequence
// itself (dual numbers), in both precisions.  The derivative formulas
// (2.10)-(2.12), applied once after a plain duplication, divide by
// differences of the arguments: they lose digits wherever two arguments are
// close (every pair at low z, most pairs of a typical batch) or where two
// roots of E^2 nearly coincide.  Measured in FP64 against the Leibniz-rule
// oracle, the formulas left d t / d theta at 2e-2 for Omega_L0 = 1e-12 (a
// near-double root at rho = 0) and d X / d Omega_r0 at 3e-5 for
// Omega_r0 = 1e-12, where the dual tangents give 5e-14 and 4e-13.  Only
// R_C's tangents use (2.10) (R_C(x, y) = R_F(x, y, y), no differences; see
// rc_value_grad).
// Phi(w) = [R_C(1, 1-w) - (1-w)^-1/2] / w: the part of R_C(y + d, y) - y^-1/2
// that is linear in w = d / (y + d), as a series for small w (coefficients
// 1/(2n+1) - C(2n,n)/4^n, n >= 1) and directly otherwise.
// The coefficients 1/(2n+1) - C(2n,n)/4^n, n = 1 .. 17 (exact rationals rounded).
#define LCDM_PHI_CS {-0.16666666666666666, -0.175, -0.16964285714285715, -0.1623263888888889,                   \
                     -0.1551846590909091, -0.14866286057692307, -0.14280598958333332, -0.13755708582261028,      \
                     -0.13283900210731908, -0.1285780043829055, -0.12470983422320822, -0.12118025779724122,      \
                     -0.1179439800756949, -0.11496322216658757, -0.11220638357823895, -0.10964690378838868,      \
                     -0.10726233098788986}
template <class S> LCDM_HD S phi_rc(const S& w, int* fail) {
    typedef typename Base<S>::type T;
    constexpr int NT = sizeof(T) == 4 ? 9 : 17;
    if (sval(vof(w)) <= cst<T>(0.1)) {
        constexpr double cs[17] = LCDM_PHI_CS;
        S acc = w * cst<T>(0.0) + cst<T>(cs[NT - 1]);
#pragma unroll
        for (int n = NT - 1; n >= 1; n--) acc = acc * w + cst<T>(cs[n - 1]);
        return acc;
    }
    S one_w = cst<T>(1.0) - w;
    S one = one_w + w;   // 1 with the type of w
    return (rc_any(one, one_w, fail) - one / ssqrt(one_w)) / w;
}

// Quartic (Or > 0).  The big root A ~ -Om/Or and the prefactor Or^-1/2 each
// depend on Or like 1/Or; their product does not.  By the homogeneity of the
// Carlson integrals (R_F, R_C ~ s^-1/2; R_J, R_D ~ s^-3/2) every argument is
// scaled by lam = Or, and the big root enters only through
//   a_A = -lam A,  m_A = lam rho_A,  eps_A = -1/rho_A,  rho_A = 1 + A,
// so that X~_A = sqrt(lam (z - A)) = sqrt(lam z + a_A), Y~_A = sqrt(a_A) and
// every factor below has derivatives of its own size.  Written out:
//   eq. (3.7):  chi H0/c = 2z R_F(u~^2)
//   eq. (3.8):  t H0 = 2z [ R_C(k s5, k q5) - eps_A R_F - z^2/3 m_A (1 + eps_A rho_B) |1 + eps_A rho_P|^2 R_J(u~^2, lam u_A5^2) ]
//   eq. (3.9):  X H0/c = z [ T0 + (2 rho_B^2 - |P-B|^2) R_F + rho_A G ]
// with u~ = sqrt(lam) u and the terms defined in the code.
template <class S, class PS, bool WT, bool WX>
LCDM_HD void quartic_integrals(typename Base<S>::type z, const S& lam, const S& aA, const S& mA, const S& epsA,
                               const S& rhoA, const S& B, const PS& P, const S& YB, const PS& YP, const S& qA,
                               const S& qB, const PS& wP, const S& nrm, S& Ichi, S& It, S& IX, int* fail) {
    typedef typename Base<S>::type T;
    const T one = cst<T>(1.0), third = cst<T>(1.0 / 3.0);
    const T z2 = z * z;
    S XtA = ssqrt(lam * z + aA), YtA = ssqrt(aA);
    S XB = ssqrt(z - B);
    PS XP = psqrt(prsub(z, P));
    S ppYP = pprod(YP), ppXP = pprod(XP);
    // u_ij of Sec. 3.1 with z1 = 0, times sqrt(lam): u_AB (real), pair (u_AP, u_AP*),
    // written with the ratios n_j = X_j / Y_j = sqrt(1 + z q_j), q_j = -1/r_j:
    //   u_AB = N (n_A n_B + n_P n_P*),  u_AP = N (n_P n_A + n_P* n_B),
    // N = Y~_A Y_B |Y_P|^2 = sqrt(E^2(0)).  The tangents of n_j are z dq_j / (2 n_j),
    // so the arguments' tangents vanish with z without cancellation.
    // (wP = 1 + z q_P is formed by the caller: it cancels near z = Re r_P)
    S nA = ssqrt(one + qA * z), nB = ssqrt(one + qB * z);
    PS nP = psqrt(wP);
    S uAB = nrm * (nA * nB + pprod(nP));
    PS uAP = pscale(pscale(nP, nA) + pscale(pswap(nP), nB), nrm);
    S x1 = uAB * uAB;
    S rhoB = B + one;
    PS rhoP = padd(P, one);
    S ppPA = pprod(padd(pscale(rhoP, epsA), one));     // |P - A|^2 / rho_A^2
    S ppPB = pprod(padd(P, -B));
    enum { NJ = (WT ? 1 : 0) + (WX ? 1 : 0) };
    S p[NJ > 0 ? NJ : 1];
    int jt = 0, jx = WT ? 1 : 0;
    if (WT) p[jt] = -(mA * ppPA * rhoB * z2);          // lam u_A5^2 - x1
    if (WX) p[jx] = -(lam * ppPB * z2);                // lam u_B0^2 - x1
    // eq. (3.8), i = A: everything but the R_F and R_J terms before the
    // duplication sequence, so that only three factors stay live across it
    S RCp, kB, cJ;
    if (WT) {
        // R_C(s_A5^2, q_A5^2) scaled by eps_A (homogeneity) is R_C(k s5, k q5) =
        // k^-1/2 R_C(s5, q5) with k = (1+z) / cA, cA = (1 + eps_A)(1 + eps_A (1+z)).
        // The part of k^-1/2 linear in eps_A is combined with -eps_A R_F: the two
        // cancel as z -> 0, and so do their tangents, which carry
        // d eps_A / d Or ~ 1 / Om.  With sqrt(cA) - 1 = eps_A (2 + z + eps_A (1+z)) / (sqrt(cA) + 1):
        //   R_C(k s5, k q5) - eps_A R_F = RC' + eps_A [RC' (2 + z + eps_A (1+z)) / (sqrt(cA) + 1) - R_F],
        // RC' = (1+z)^-1/2 R_C(s5, q5), and the bracket is O(z).
        const T izh = one / ssqrt(one + z);
        S cA = (one + epsA) * (one + epsA * (one + z));
        S q5 = x1 + p[jt];
        S s5 = q5 + mA * pprod(rhoP) * rhoB * z2 * cA * (izh * izh);
        RCp = rc_any(s5, q5, fail) * izh;
        kB = (cst<T>(2.0) + z + epsA * (one + z)) / (ssqrt(cA) + one);
        cJ = mA * (one + epsA * rhoB) * ppPA * (z2 * third);
    }
    S RF, RD1, RJ[NJ > 0 ? NJ : 1], DJ;
    carlson_any<NJ, WX, WX>(uAB, uAP, p, RF, RD1, RJ, fail, &DJ);
    Ichi = RF * (z + z);                               // eq. (3.7)
    if (WT) {
        S Bk = RCp * kB - RF;
        It = (RCp + epsA * Bk - cJ * RJ[jt]) * (z + z);
    }
    if (WX) {                                          // eq. (3.9), i = B, l = A
        // The l = A part of (3.9), rho_A G, is a sum of O(1) terms that cancel to
        // O(lam): written out so that every term is O(1) by itself:
        //   G1 + G4 = z^2/3 |P-B|^2 [c (a_A + lam B) h0 Delta_J + E1 R_D1],
        //   G2 + G3 = c [R_C(y + d, y) - y^-1/2] + c Y_B X_B Num / (...) + E1 Y_B X_B / (X~_A Y~_A u~),
        // with h0 = -lam z^2 |P-B|^2, Delta_J = (R_J(x1 + h0) - R_D) / h0, y = lam q_B0^2,
        // d = lam z^2, E1 and Num exact polynomials carrying a factor lam, and
        // c = 1 - eps_A (rho_B + rho_P + rho_P*).
        S p0 = x1 + p[jx];                                    // lam u_B0^2
        S y = p0 / (YB * YB * XB * XB);                       // lam q_B0^2
        S dl = lam * z2;                                      // lam (s_B0^2 - q_B0^2)
        S yd = y + dl;
        S Phi = phi_rc(dl / yd, fail);
        S eB = one / (XB + YB);
        PS XY = XP + YP;
        S Dpp = psum(prcp(XY) * pswap(XY)) * cst<T>(0.5);
        // [X_B X_P X_P* / X_A]_0^z / z, telescoped, times Or^-1/2
        S T0 = (eB * ppXP + YB * Dpp) / XtA - lam * YB * ppYP / ((XtA + YtA) * XtA * YtA);
        S T1 = (rhoB * rhoB * cst<T>(2.0) - ppPB) * RF;
        S Srho = psum(rhoP), Qrho = pprod(rhoP);
        S c = one - epsA * (rhoB + Srho);
        S aB = aA + lam * B;
        S rE1 = -(mA * (Srho * cst<T>(2.0) + epsA * (Qrho + rhoB * rhoB + rhoB * Srho)));   // rho_A E1
        S XYu = XtA * YtA * uAB;
        S sp0 = ssqrt(p0);
        S rNum = mA * (x1 * (aA * (z - B * cst<T>(2.0)) - lam * B * B) + aB * aB * ppPB * z2);   // rho_A Num
        S rPart1 = mA * z2 / yd * Phi / ssqrt(yd);            // rho_A [R_C(y+d, y) - y^-1/2]
        S rG = ppPB * (z2 * third) * (rE1 * RD1 - c * aB * mA * ppPB * DJ * z2)
               + c * rPart1 + c * YB * XB * rNum / (sp0 * XYu * (XYu + aB * sp0)) + rE1 * XB * YB / XYu;
        IX = (T0 + T1 + rG) * z;
    }
}

template <class S, class PS, bool WT, bool WX>
LCDM_HD void cubic_integrals(typename Base<S>::type z, const S& A, const PS& P, const S& YA, const PS& YP,
                             const S& amh, const S& qA, const PS& wP, const S& nrm, S& Ichi, S& It, S& IX,
                             int* fail) {
    typedef typename Base<S>::type T;
    const T one = cst<T>(1.0);
    const T z2 = z * z;
    S XA = ssqrt(z - A);
    PS XP = psqrt(prsub(z, P));
    S ppYP = pprod(YP), ppXP = pprod(XP);
    // u_i of App. B.1 with z1 = 0: u_A (real) and the pair (u_P, u_P*), from the
    // ratios n_j = X_j / Y_j = sqrt(1 + z q_j) as in the quartic:
    //   u_A = N (n_A + n_P n_P*),  u_P = N (n_P + n_P* n_A),  N = Y_A |Y_P|^2
    S nA = ssqrt(one + qA * z);
    PS nP = psqrt(wP);   // wP = 1 + z q_P, formed by the caller
    S uA = nrm * (nA + pprod(nP));
    PS uP = pscale(nP + pscale(pswap(nP), nA), nrm);
    S x1 = uA * uA;
    enum { NJ = WT ? 1 : 0 };
    S p[1];
    S rhoA = A + one;
    if (WT) p[0] = rhoA * z2;                          // u_A5^2 - x1
    S RC5;                                             // eq. (B.2)'s R_C term, before the duplication
    if (WT) {
        S s5 = YA * ppYP * (one + z) + XA * ppXP;
        S q5 = (x1 + p[0]) * (one + z);
        RC5 = rc_any(s5 * s5, q5, fail);
    }
    S RF, RD1, RJ[1];
    carlson_any<NJ, WX, false>(uA, uP, p, RF, RD1, RJ, fail);
    Ichi = amh * RF * (z + z);                         // eq. (B.1)
    if (WT) It = amh * (z + z) * (RJ[0] * (z2 * cst<T>(1.0 / 3.0)) + RC5);   // eq. (B.2)
    if (WX) {                                          // eq. (B.3), i = A
        S ppPA = pprod(padd(P, -A));
        S eA = one / (XA + YA);
        PS XY = XP + YP;
        S Dpp = psum(prcp(XY) * pswap(XY)) * cst<T>(0.5);
        S T0 = eA * ppXP + YA * Dpp;                   // [X_A X_P X_P*]_0^z / z
        S T1 = (rhoA * rhoA * cst<T>(3.0) - ppPA) * RF;
        S T2 = (A + psum(P) + cst<T>(3.0)) * (ppPA * RD1 * (z2 * cst<T>(1.0 / 3.0)) + YA * XA / uA) * cst<T>(2.0);
        IX = amh * (T0 + T1 + T2) * (z + z) * cst<T>(1.0 / 3.0);
    }
}

// The same integrals as one real call, for the kernels whose tangents or
// outputs need more registers than the inlined path can hold (seven-column
// tangents, X's tangents): there the allocator handles the pair in two parts.
template <class S, class PS, bool WT, bool WX>
LCDM_NI void quartic_integrals_call(typename Base<S>::type z, const S& lam, const S& aA, const S& mA, const S& epsA,
                                    const S& rhoA, const S& B, const PS& P, const S& YB, const PS& YP, const S& qA,
                                    const S& qB, const PS& wP, const S& nrm, S& Ichi, S& It, S& IX, int* fail) {
    quartic_integrals<S, PS, WT, WX>(z, lam, aA, mA, epsA, rhoA, B, P, YB, YP, qA, qB, wP, nrm, Ichi, It, IX, fail);
}
template <class S, class PS, bool WT, bool WX>
LCDM_NI void cubic_integrals_call(typename Base<S>::type z, const S& A, const PS& P, const S& YA, const PS& YP,
                                  const S& amh, const S& qA, const PS& wP, const S& nrm, S& Ichi, S& It, S& IX,
                                  int* fail) {
    cubic_integrals<S, PS, WT, WX>(z, A, P, YA, YP, amh, qA, wP, nrm, Ichi, It, IX, fail);
}

template <bool CALL, class S, class PS, bool WT, bool WX>
LCDM_HD void quartic_integrals_any(typename Base<S>::type z, const S& lam, const S& aA, const S& mA, const S& epsA,
                                   const S& rhoA, const S& B, const PS& P, const S& YB, const PS& YP, const S& qA,
                                   const S& qB, const PS& wP, const S& nrm, S& Ichi, S& It, S& IX, int* fail) {
    if constexpr (CALL)
        quartic_integrals_call<S, PS, WT, WX>(z, lam, aA, mA, epsA, rhoA, B, P, YB, YP, qA, qB, wP, nrm, Ichi, It, IX, fail);
    else
        quartic_integrals<S, PS, WT, WX>(z, lam, aA, mA, epsA, rhoA, B, P, YB, YP, qA, qB, wP, nrm, Ichi, It, IX, fail);
}
template <bool CALL, class S, class PS, bool WT, bool WX>
LCDM_HD void cubic_integrals_any(typename Base<S>::type z, const S& A, const PS& P, const S& YA, const PS& YP,
                                 const S& amh, const S& qA, const PS& wP, const S& nrm, S& Ichi, S& It, S& IX,
                                 int* fail) {
    if constexpr (CALL) cubic_integrals_call<S, PS, WT, WX>(z, A, P, YA, YP, amh, qA, wP, nrm, Ichi, It, IX, fail);
    else cubic_integrals<S, PS, WT, WX>(z, A, P, YA, YP, amh, qA, wP, nrm, Ichi, It, IX, fail);
}

// ------------------------------------------------------ z -> infinity ------
// The upper limit at infinity (Sec. 2.1.1: the age t(0, inf); the comoving
// distance to the particle horizon chi(0, inf)) of the quantities above, with
// the same root labels and scalings.  As z grows, n_j / sqrt(z) -> sqrt(q_j),
// every u grows like z, and with the homogeneity of R_F, R_C (degree -1/2)
// and R_J (degree -3/2) every power of z cancels; in eq. (3.8)
// (1+z) / (1 + eps_A (1+z)) -> 1 / eps_A.  In (B.2) the R_C term falls off
// like z^-1/2 and drops out.  Ichi and It are in the units of their
// finite-z counterparts (c/H0 and 1/H0 after the record's prefactors).
template <class S, class PS>
LCDM_NI void quartic_limits(const S& mA, const S& epsA, const S& B, const PS& P, const S& qA, const S& qB,
                            const PS& qP, const S& nrm, S& Ichi, S& It, int* fail) {
    typedef typename Base<S>::type T;
    const T one = cst<T>(1.0), third = cst<T>(1.0 / 3.0);
    S nA = ssqrt(qA), nB = ssqrt(qB);
    PS nP = psqrt(qP);
    S uAB = nrm * (nA * nB + pprod(nP));
    PS uAP = pscale(pscale(nP, nA) + pscale(pswap(nP), nB), nrm);
    S x1 = uAB * uAB;
    S rhoB = B + one;
    PS rhoP = padd(P, one);
    S ppPA = pprod(padd(pscale(rhoP, epsA), one));
    S p[1];
    p[0] = -(mA * ppPA * rhoB);
    S RF, RD1, RJ[1];
    carlson_any<1, false, false>(uAB, uAP, p, RF, RD1, RJ, fail);
    Ichi = RF * cst<T>(2.0);                                   // eq. (3.7), z -> inf
    S kq5 = (x1 + p[0]) / ((one + epsA) * epsA);
    S ks5 = kq5 + mA * pprod(rhoP) * rhoB;
    It = (rc_any(ks5, kq5, fail) - epsA * RF - mA * (one + epsA * rhoB) * ppPA * RJ[0] * third)
         * cst<T>(2.0);                                        // eq. (3.8), z -> inf
}

template <class S, class PS>
LCDM_NI void cubic_limits(const S& A, const S& amh, const S& qA, const PS& qP, const S& nrm, S& Ichi, S& It,
                          int* fail) {
    typedef typename Base<S>::type T;
    const T one = cst<T>(1.0);
    S nA = ssqrt(qA);
    PS nP = psqrt(qP);
    // u_A / z -> N n_P n_P*,  u_P / z -> N n_P* n_A  (the plain u_i -> Y_i = sqrt(-r_i))
    S uA = nrm * pprod(nP);
    PS uP = pscale(pswap(nP), nA * nrm);
    S p[1];
    p[0] = A + one;                                            // u_A5^2 - u_A^2 = rho_A
    S RF, RD1, RJ[1];
    carlson_any<1, false, false>(uA, uP, p, RF, RD1, RJ, fail);
    Ichi = amh * RF * cst<T>(2.0);                             // eq. (B.1), z -> inf
    It = amh * RJ[0] * cst<T>(2.0 / 3.0);                      // eq. (B.2), z -> inf
}

}  // namespace lcdm
