// Distance assembly for one (cosmology, redshift) pair, written once for any
// scalar S: a plain number (values only) or Dual<T,K> (values and tangents
// with respect to the density parameters).
//
// Carlson integrals enter through carlson_any / rc_any.  Their tangents use
//   dR_F/dx_m = -R_D(..x_m..)/6                                (eq. 2.10)
//   dR_J/dx_m = (R_J - R_D(..x_m..)) / (2 (p - x_m))            (eq. 2.11)
//   dR_J/dp   = 3/2 { (p^2 R_F - 2 p R_G + sqrt(x1 x2 x3))
//                     / (p prod(p - x_i)) - sum 1/(p - x_i) R_J/3 } (eq. 2.12,
//               with R_G(x1,x2,x3) where the printed formula shows R_D; R_G is
//               formed from the three R_D by 6 R_G = sum_m x_m (e1 - x_m) R_D_m)
// and, for R_D itself, dR_D(x,y,z)/dx = (R_D(x,y,z) - R_D(y,z,x)) / (2 (z - x))
// with the special-argument derivative from homogeneity (degree -3/2).  All
// R_D, R_J and R_F values come from one shared duplication sequence.
//
// Cauchy principal values (Sec. 2.2) for negative p or y:
//   (q+z) R_J(x,y,z,-q) = (s-z) R_J(x,y,z,s) - 3 R_F + 3 sqrt(xyz/(xy+sq)) R_C(xy+sq, sq),
//   s = (z(x+y+q) - xy)/(z+q), z the real member of the triple;
//   R_C(x, -q) = sqrt(x/(x+q)) R_C(x+q, q).
#pragma once
#include "lcdm_math.cuh"

namespace lcdm {

template <class P> struct PairVal;
template <class T, int K> struct PairVal<CPair<Dual<T, K> > > { typedef CPair<T> type; };
template <class T, int K> struct PairVal<RPair<Dual<T, K> > > { typedef RPair<T> type; };

// ---------------------------------------------------------------- values ----
template <class T> LCDM_HD T rc_any(T x, T y, int* fail) {
    if (sval(y) < 0) {
        T x2 = x - y, y2 = -y;
        return ssqrt(x / x2) * rc_value(x2, y2, fail);
    }
    return rc_value(x, y, fail);
}

template <int NJ, class T, class PT>
LCDM_HD void carlson_any(T x1, PT pr, const T* p, bool needRD1, T& RF, T& RD1, T* RJ, int* fail) {
    T tr[NJ > 0 ? NJ : 1], s[NJ > 0 ? NJ : 1], q[NJ > 0 ? NJ : 1];
    bool pv[NJ > 0 ? NJ : 1];
#pragma unroll
    for (int j = 0; j < NJ; j++) {
        pv[j] = sval(p[j]) < 0;
        if (pv[j]) {
            q[j] = -p[j];
            s[j] = (x1 * (psum(pr) + q[j]) - pprod(pr)) / (x1 + q[j]);
            if (!(sval(s[j]) > 0)) *fail = 2;
            tr[j] = s[j];
        } else {
            tr[j] = p[j];
        }
    }
    if (needRD1) {
        DupResult<T, NJ, PT> R = carlson_dup<T, NJ, true>(x1, pr, tr, fail);
        RF = R.RF; RD1 = R.RD1;
#pragma unroll
        for (int j = 0; j < NJ; j++) RJ[j] = R.RJ[j];
    } else {
        DupResult<T, NJ, PT> R = carlson_dup<T, NJ, false>(x1, pr, tr, fail);
        RF = R.RF; RD1 = RF;
#pragma unroll
        for (int j = 0; j < NJ; j++) RJ[j] = R.RJ[j];
    }
#pragma unroll
    for (int j = 0; j < NJ; j++) {
        if (pv[j]) {
            T xy = pprod(pr), sq = s[j] * q[j];
            T rc = rc_value(xy + sq, sq, fail);
            RJ[j] = ((s[j] - x1) * RJ[j] - cst<T>(3.0) * RF + cst<T>(3.0) * ssqrt(x1 * xy / (xy + sq)) * rc)
                    / (q[j] + x1);
        }
    }
}

// --------------------------------------------------------------- tangents ---
template <class T, int K> LCDM_HD Dual<T, K> rc_dual_pos(const Dual<T, K>& x, const Dual<T, K>& y, int* fail) {
    DupResult<T, 0, RPair<T> > R = carlson_dup<T, 0, true>(x.v, mkrp<T>(y.v, y.v), (const T*)0, fail);
    // R_C(x,y) = R_F(x,y,y): dR_C/dx = -R_D(y,y,x)/6, dR_C/dy = -(2 R_D(x,y,y))/6   (eqs. 2.8, 2.10)
    T gx = R.RD1 * cst<T>(-1.0 / 6.0), gy = (R.RDp.a + R.RDp.b) * cst<T>(-1.0 / 6.0);
    Dual<T, K> r;
    r.v = R.RF;
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = gx * x.d[k] + gy * y.d[k];
    return r;
}
template <class T, int K> LCDM_HD Dual<T, K> rc_any(const Dual<T, K>& x, const Dual<T, K>& y, int* fail) {
    if (sval(y.v) < 0) {
        Dual<T, K> x2 = x - y, y2 = -y;
        return ssqrt(x / x2) * rc_dual_pos(x2, y2, fail);
    }
    return rc_dual_pos(x, y, fail);
}

template <int NJ, class T, int K, class PD>
LCDM_HD void carlson_any(const Dual<T, K>& x1, const PD& pr, const Dual<T, K>* p, bool needRD1, Dual<T, K>& RF,
                         Dual<T, K>& RD1, Dual<T, K>* RJ, int* fail) {
    typedef Dual<T, K> D;
    typedef typename PairVal<PD>::type PT;
    const T xv = x1.v;
    const PT prv = pval(pr);
    D tr[NJ > 0 ? NJ : 1], s[NJ > 0 ? NJ : 1], q[NJ > 0 ? NJ : 1];
    T trv[NJ > 0 ? NJ : 1];
    bool pv[NJ > 0 ? NJ : 1];
#pragma unroll
    for (int j = 0; j < NJ; j++) {
        pv[j] = sval(p[j].v) < 0;
        if (pv[j]) {
            q[j] = -p[j];
            s[j] = (x1 * (psum(pr) + q[j]) - pprod(pr)) / (x1 + q[j]);
            if (!(sval(s[j].v) > 0)) *fail = 2;
            tr[j] = s[j];
        } else {
            tr[j] = p[j];
        }
        trv[j] = tr[j].v;
    }
    DupResult<T, NJ, PT> R = carlson_dup<T, NJ, true>(xv, prv, trv, fail);
    // R_F, eq. (2.10)
    RF.v = R.RF;
#pragma unroll
    for (int k = 0; k < K; k++) RF.d[k] = (R.RD1 * x1.d[k] + pdot_k(R.RDp, pr, k)) * cst<T>(-1.0 / 6.0);
    // R_D(x2, x3, x1)
    if (needRD1) {
        PT dpair = pscale(prsub(R.RD1, R.RDp) / prsub(xv, prv), cst<T>(0.5));
        T d1 = (cst<T>(-1.5) * R.RD1 - pdot(prv, dpair)) / xv;
        RD1.v = R.RD1;
#pragma unroll
        for (int k = 0; k < K; k++) RD1.d[k] = d1 * x1.d[k] + pdot_k(dpair, pr, k);
    }
    if (NJ > 0) {
        // 6 R_G = sum_m x_m (e1 - x_m) R_D_m
        T RG = (xv * psum(prv) * R.RD1 + pdot(R.RDp, prv * padd(pswap(prv), xv))) * cst<T>(1.0 / 6.0);
        T sq3 = ssqrt(xv) * pprod(psqrt(prv));
#pragma unroll
        for (int j = 0; j < NJ; j++) {
            const T pt = trv[j], J = R.RJ[j];
            const T ipx = cst<T>(1.0) / (pt - xv);
            const PT ipp = prcp(prsub(pt, prv));
            T d1 = (J - R.RD1) * ipx * cst<T>(0.5);
            PT dpair = pscale(prsub(J, R.RDp) * ipp, cst<T>(0.5));
            T dp = cst<T>(1.5) * ((pt * pt * R.RF - cst<T>(2.0) * pt * RG + sq3) * ipx * pprod(ipp) / pt
                                  - (ipx + psum(ipp)) * J * cst<T>(1.0 / 3.0));
            D Jd;
            Jd.v = J;
#pragma unroll
            for (int k = 0; k < K; k++) Jd.d[k] = d1 * x1.d[k] + pdot_k(dpair, pr, k) + dp * tr[j].d[k];
            if (!pv[j]) {
                RJ[j] = Jd;
            } else {
                D xy = pprod(pr), sq = s[j] * q[j];
                D rc = rc_dual_pos(xy + sq, sq, fail);
                RJ[j] = ((s[j] - x1) * Jd - RF * cst<T>(3.0) + ssqrt(x1 * xy / (xy + sq)) * rc * cst<T>(3.0))
                        / (q[j] + x1);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Distance integrals, dimensionless: I_chi = chi H0/c, I_t = t H0, I_X = X H0/c,
// each including the alpha_m^-1/2 prefactor.  z1 = 0, z2 = z.
// Roots in z: A (real), B (real, quartic only), the pair P; Y = sqrt(-root).
// Labels: t uses i = A; X uses i = B, l = A (quartic) or i = A (cubic); the
// pair members are j, k.  See eqs. (3.7)-(3.9) and (B.1)-(B.3).
// ---------------------------------------------------------------------------
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
LCDM_NI void quartic_integrals(typename Base<S>::type z, const S& lam, const S& aA, const S& mA, const S& epsA,
                               const S& rhoA, const S& B, const PS& P, const S& YB, const PS& YP, S& Ichi, S& It,
                               S& IX, int* fail) {
    typedef typename Base<S>::type T;
    const T one = cst<T>(1.0), third = cst<T>(1.0 / 3.0);
    const T z2 = z * z;
    S XtA = ssqrt(lam * z + aA), YtA = ssqrt(aA);
    S XB = ssqrt(z - B);
    PS XP = psqrt(prsub(z, P));
    S ppYP = pprod(YP), ppXP = pprod(XP);
    // u_ij of Sec. 3.1 with z1 = 0, times sqrt(lam): u_AB (real), pair (u_AP, u_AP*)
    S uAB = XtA * XB * ppYP + YtA * YB * ppXP;
    PS W = XP * pswap(YP);
    PS uAP = pscale(W, XtA * YB) + pscale(pswap(W), YtA * XB);
    S x1 = uAB * uAB;
    PS pr = uAP * uAP;
    S rhoB = B + one;
    PS rhoP = padd(P, one);
    S ppPA = pprod(padd(pscale(rhoP, epsA), one));     // |P - A|^2 / rho_A^2
    S ppPB = pprod(padd(P, -B));
    enum { NJ = (WT ? 1 : 0) + (WX ? 1 : 0) };
    S p[NJ > 0 ? NJ : 1];
    int jt = 0, jx = WT ? 1 : 0;
    if (WT) p[jt] = x1 - mA * ppPA * rhoB * z2;        // lam u_A5^2
    if (WX) p[jx] = x1 - lam * ppPB * z2;              // lam u_B0^2
    S RF, RD1, RJ[NJ > 0 ? NJ : 1];
    carlson_any<NJ>(x1, pr, p, WX, RF, RD1, RJ, fail);
    Ichi = RF * (z + z);                               // eq. (3.7)
    if (WT) {                                          // eq. (3.8), i = A
        S kq5 = p[jt] * (one + z) / ((one + epsA) * (one + epsA * (one + z)));
        S ks5 = kq5 + mA * pprod(rhoP) * rhoB * z2;
        It = (rc_any(ks5, kq5, fail) - epsA * RF - mA * (one + epsA * rhoB) * ppPA * RJ[jt] * (z2 * third)) * (z + z);
    }
    if (WX) {                                          // eq. (3.9), i = B, l = A
        S lq0 = p[jx] / (YB * YB * XB * XB);
        S ls0 = lq0 + lam * z2;
        S eB = one / (XB + YB);
        PS XY = XP + YP;
        S Dpp = psum(prcp(XY) * pswap(XY)) * cst<T>(0.5);
        // [X_B X_P X_P* / X_A]_0^z / z, telescoped, times Or^-1/2
        S T0 = (eB * ppXP + YB * Dpp) / XtA - lam * YB * ppYP / ((XtA + YtA) * XtA * YtA);
        S T1 = (rhoB * rhoB * cst<T>(2.0) - ppPB) * RF;
        S G = mA * ppPA * (ppPB * RD1 * (z2 * third) + XB * YB / (XtA * YtA * uAB))
              + (one - epsA * (rhoB + psum(rhoP))) * (rc_any(ls0, lq0, fail) + ppPB * (aA + lam * B) * RJ[jx] * (z2 * third));
        IX = (T0 + T1 + rhoA * G) * z;
    }
}

template <class S, class PS, bool WT, bool WX>
LCDM_NI void cubic_integrals(typename Base<S>::type z, const S& A, const PS& P, const S& YA, const PS& YP,
                             const S& amh, S& Ichi, S& It, S& IX, int* fail) {
    typedef typename Base<S>::type T;
    const T one = cst<T>(1.0);
    const T z2 = z * z;
    S XA = ssqrt(z - A);
    PS XP = psqrt(prsub(z, P));
    S ppYP = pprod(YP), ppXP = pprod(XP);
    // u_i of App. B.1 with z1 = 0: u_A (real) and the pair (u_P, u_P*)
    S uA = XA * ppYP + YA * ppXP;
    PS W = XP * pswap(YP);
    PS uP = pscale(W, YA) + pscale(pswap(W), XA);
    S x1 = uA * uA;
    PS pr = uP * uP;
    enum { NJ = WT ? 1 : 0 };
    S p[1];
    S rhoA = A + one;
    if (WT) p[0] = x1 + rhoA * z2;                     // u_A5^2
    S RF, RD1, RJ[1];
    carlson_any<NJ>(x1, pr, p, WX, RF, RD1, RJ, fail);
    Ichi = amh * RF * (z + z);                         // eq. (B.1)
    if (WT) {                                          // eq. (B.2)
        S s5 = YA * ppYP * (one + z) + XA * ppXP;
        S q5 = p[0] * (one + z);
        It = amh * (z + z) * (RJ[0] * (z2 * cst<T>(1.0 / 3.0)) + rc_any(s5 * s5, q5, fail));
    }
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

}  // namespace lcdm
