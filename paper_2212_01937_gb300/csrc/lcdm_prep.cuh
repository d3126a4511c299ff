// Root preparation, one or four lanes per cosmology, FP64: factorise E^2 (eq. 3.2),
// classify the roots, choose the root labels, precompute the per-cosmology
// constants and the root tangents (App. A, eqs. A.1-A.4).
#pragma once
#include "lcdm_kernels.cuh"

namespace lcdm {

// ---------------------------------------------------------------- roots -----
struct cd { double re, im; };
LCDM_HD cd cmk(double r, double i) { cd c; c.re = r; c.im = i; return c; }
LCDM_HD cd cadd(cd a, cd b) { return cmk(a.re + b.re, a.im + b.im); }
LCDM_HD cd csub(cd a, cd b) { return cmk(a.re - b.re, a.im - b.im); }
LCDM_HD cd cmul(cd a, cd b) { return cmk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
// One copy of the double-precision division for all of the preparation: each
// '/' would otherwise carry its own copy of the division's slow path.
LCDM_NI double ddiv(double a, double b) { return a / b; }

LCDM_HD cd cdiv(cd a, cd b) {
    double s = fabs(b.re) > fabs(b.im) ? fabs(b.re) : fabs(b.im);
    double is = ddiv(1.0, s);
    double br = b.re * is, bi = b.im * is, inv = ddiv(is, br * br + bi * bi);
    return cmk((a.re * br + a.im * bi) * inv, (a.im * br - a.re * bi) * inv);
}
LCDM_HD double cabs_(cd a) { return hypot(a.re, a.im); }
LCDM_HD cd csqrt_(cd a) {
    double r = cabs_(a);
    if (a.re >= 0) { double t = sqrt(0.5 * (r + a.re)); return cmk(t, t > 0 ? a.im * ddiv(0.5, t) : 0.0); }
    double t = sqrt(0.5 * (r - a.re));
    return cmk(fabs(a.im) * ddiv(0.5, t), a.im < 0 ? -t : t);
}

LCDM_HD double cnorm(cd a) { return a.re * a.re + a.im * a.im; }
// 1/b with one real division (the polynomial's values stay far inside the
// double range for the normalised coefficients used here)
LCDM_HD cd crcp(cd b) {
    double s = ddiv(1.0, cnorm(b));
    return cmk(b.re * s, -b.im * s);
}

// p(x) = sum_k c[k] x^k (degree n, c[n] = 1) and p'(x) by Horner's rule
LCDM_HD void horner(const double* c, int n, cd x, cd& p, cd& dp) {
    p = cmk(c[n], 0); dp = cmk(0, 0);
#pragma unroll 1
    for (int k = n - 1; k >= 0; k--) { dp = cadd(cmul(dp, x), p); p = cadd(cmul(p, x), cmk(c[k], 0)); }
}

// Error-free transformations: Knuth's sum, and the product by the fused
// multiply-add (a b = p + e exactly).
LCDM_HD void two_sum_d(double a, double b, double& s, double& e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
LCDM_HD void two_prod_d(double a, double b, double& p, double& e) {
    p = a * b;
    e = fma(a, b, -p);
}

// p(x) = sum_k a[k] x^k (degree n) and p'(x) at complex x by the compensated
// Horner scheme (Graillat, Langlois and Louvet): the rounding error of every
// Horner step is carried, exactly, into a second Horner recurrence, so the
// value is as accurate as if it had been evaluated in twice the working
// precision.  Newton's method on it then finds a root to the last bit even
// where p' is small, as at the near-double roots of the no-Big-Bang boundary.
LCDM_HD void horner_comp(const double* a, int n, cd x, cd& p, cd& dp) {
    cd h = cmk(a[n], 0), q = cmk(0, 0);
    dp = cmk(0, 0);
#pragma unroll 1
    for (int k = n - 1; k >= 0; k--) {
        dp = cadd(cmul(dp, x), h);
        double p1, e1, p2, e2, p3, e3, p4, e4, s1, e5, s2, e6, t1, e7;
        two_prod_d(h.re, x.re, p1, e1);
        two_prod_d(h.im, x.im, p2, e2);
        two_prod_d(h.re, x.im, p3, e3);
        two_prod_d(h.im, x.re, p4, e4);
        two_sum_d(p1, -p2, s1, e5);
        two_sum_d(p3, p4, s2, e6);
        two_sum_d(s1, a[k], t1, e7);
        q = cadd(cmul(q, x), cmk(((e1 - e2) + e5) + e7, (e3 + e4) + e6));
        h = cmk(t1, s2);
    }
    p = cadd(h, q);
}

// Newton steps on the polynomial with the given (not normalised) coefficients,
// evaluated by horner_comp; a step is kept only while |p| decreases.
LCDM_HD void polish_root(const double* a, int n, cd& x) {
    cd p, dp;
    horner_comp(a, n, x, p, dp);
#pragma unroll 1
    for (int it = 0; it < 2; it++) {
        if ((dp.re == 0 && dp.im == 0) || (p.re == 0 && p.im == 0)) return;
        const cd xn = csub(x, cdiv(p, dp));
        cd pn, dpn;
        horner_comp(a, n, xn, pn, dpn);
        if (!(cnorm(pn) < cnorm(p))) return;
        x = xn; p = pn; dp = dpn;
    }
}

// Single-precision elementary functions for the starting circles only (no
// accuracy needed there): the fast hardware approximations on the device.
LCDM_HD float flog(float x) {
#ifdef __CUDA_ARCH__
    return __logf(x);
#else
    return logf(x);
#endif
}
LCDM_HD float fexp(float x) {
#ifdef __CUDA_ARCH__
    return __expf(x);
#else
    return expf(x);
#endif
}
LCDM_HD float fcos(float x) {
#ifdef __CUDA_ARCH__
    return __cosf(x);
#else
    return cosf(x);
#endif
}
LCDM_HD float fsin(float x) {
#ifdef __CUDA_ARCH__
    return __sinf(x);
#else
    return sinf(x);
#endif
}

// Starting points of the root iteration for the monic polynomial c (degree
// n <= 4): circles whose radii come from the Newton polygon of log|c_k|, so
// that a root near -Om/Or and the O(1) roots both start close.
LCDM_HD void start_points(const double* c, int n, cd* z) {
    // upper convex hull of (k, log|c_k|); single precision is enough for the start
    float lg[5];
    int idx[5], m = 0;
    for (int k = 0; k <= n; k++) lg[k] = c[k] != 0 ? flog((float)fabs(c[k])) : -1e30f;
    for (int k = 0; k <= n; k++) {
        if (c[k] == 0) continue;
        while (m >= 2) {
            int a = idx[m - 2], b = idx[m - 1];
            // remove b if it lies below the segment a-k
            if ((lg[b] - lg[a]) * (k - a) <= (lg[k] - lg[a]) * (b - a)) m--; else break;
        }
        idx[m++] = k;
    }
    int r = 0;
    for (int e = 0; e + 1 < m; e++) {
        int a = idx[e], b = idx[e + 1], w = b - a;
        float rad = fexp((lg[a] - lg[b]) / w);
        for (int j = 0; j < w && r < 4; j++) {
            float ang = 6.2831853f * j / w + 6.2831853f * a / n + 0.4f;
            z[r++] = cmk(rad * fcos(ang), rad * fsin(ang));
        }
    }
    for (; r < 4; r++) z[r] = cmk(0.5 * r + 0.1, 0.3);  // (zero constant term etc.)
}

// Roots of the monic polynomial c (degree n <= 4) by the simultaneous
// Aberth-Ehrlich iteration, G lanes per polynomial (G = 1 or 4): lane s of a
// group of G consecutive lanes owns roots s, s + G, ... and reads the others'
// current values by shuffles.  Four lanes cut the dependent chain of one
// cosmology (few cosmologies: latency-bound); one lane does no repeated work
// (many cosmologies: bound by the FP64 pipe).  Every lane of the warp must
// call this (groups with active == false take part in the shuffles without
// updating).  Single precision first, to about 1e-6 relative (short latency
// chains), then double precision from there (cubic convergence: two or three
// sweeps), stopping after a sweep with every correction below 1e-15 relative
// or once the corrections stop shrinking (rounding level of a near-multiple
// root); one Newton step per root at the end.  On return every lane of the
// group holds all n roots in z.
template <int G> __device__ void group_roots(const double* c, const double* alpha, int n, bool active, cd* z) {
    constexpr int R = 4 / G;   // roots per lane
    const unsigned full = 0xffffffffu;
    const int s = threadIdx.x & (G - 1);
    cd z0[4];
    start_points(c, n, z0);
    double zre[R], zim[R];
#pragma unroll
    for (int r = 0; r < R; r++) { zre[r] = z0[r * G + s].re; zim[r] = z0[r * G + s].im; }
    {
        float cf[5];
        for (int k = 0; k <= 4; k++) cf[k] = k <= n ? (float)c[k] : 0.f;
        float zr[R], zi[R];
#pragma unroll
        for (int r = 0; r < R; r++) { zr[r] = (float)zre[r]; zi[r] = (float)zim[r]; }
        bool done = !active;
#pragma unroll 1
        for (int itf = 0; itf < 100; itf++) {
            float ar[4], ai[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                ar[k] = G == 1 ? zr[k / G] : __shfl_sync(full, zr[k / G], k % G, G);
                ai[k] = G == 1 ? zi[k / G] : __shfl_sync(full, zi[k / G], k % G, G);
            }
            int small = 1;
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int j = r * G + s;
                if (done || j >= n) continue;
                const float xr0 = ar[j], xi0 = ai[j];
                float pr = cf[n], pi = 0.f, dr = 0.f, di = 0.f;
#pragma unroll 1
                for (int k = n - 1; k >= 0; k--) {
                    float ndr = dr * xr0 - di * xi0 + pr, ndi = dr * xi0 + di * xr0 + pi;
                    float npr = pr * xr0 - pi * xi0 + cf[k], npi = pr * xi0 + pi * xr0;
                    dr = ndr; di = ndi; pr = npr; pi = npi;
                }
                float dn = dr * dr + di * di;
                if ((pr == 0.f && pi == 0.f) || !(dn > 0.f)) continue;
                float idn = 1.0f / dn;
                float rr = (pr * dr + pi * di) * idn, ri = (pi * dr - pr * di) * idn;   // p / p'
                float sr = 0.f, si = 0.f;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    if (k == j || k >= n) continue;
                    float xr = xr0 - ar[k], xi = xi0 - ai[k], x2 = xr * xr + xi * xi;
                    if (!(x2 > 0.f)) continue;
                    float ix = 1.0f / x2;
                    sr += xr * ix; si -= xi * ix;
                }
                float qr = 1.f - (rr * sr - ri * si), qi = -(rr * si + ri * sr);
                float qn = qr * qr + qi * qi;
                if (!(qn > 0.f)) continue;
                float iq = 1.0f / qn;
                float wr = (rr * qr + ri * qi) * iq, wi = (ri * qr - rr * qi) * iq;
                zr[r] = xr0 - wr; zi[r] = xi0 - wi;
                if (!(wr * wr + wi * wi < 1e-12f * (zr[r] * zr[r] + zi[r] * zi[r]) + 1e-30f)) small = 0;
            }
            if (G > 1) {
                small &= __shfl_xor_sync(full, small, 1, G);
                small &= __shfl_xor_sync(full, small, 2, G);
            }
            if (small) done = true;
            if (__all_sync(full, done)) break;
        }
#pragma unroll
        for (int r = 0; r < R; r++)
            if (isfinite(zr[r]) && isfinite(zi[r])) { zre[r] = zr[r]; zim[r] = zi[r]; }
    }
    // Single precision can merge a complex pair of nearly double roots (near
    // the no-Big-Bang boundary) into two points on or near the real axis, and
    // for a real polynomial the iteration keeps real approximations real.
    // Two such approximations within 1e-3 of each other get imaginary
    // offsets of opposite sign (far above double precision, far below the
    // spacing), which lets the double-precision sweeps move them back into
    // the complex plane if the roots are complex; real ones return to the axis.
    {
        double cr[4], ci[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            cr[k] = G == 1 ? zre[k / G] : __shfl_sync(full, zre[k / G], k % G, G);
            ci[k] = G == 1 ? zim[k / G] : __shfl_sync(full, zim[k / G], k % G, G);
        }
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int j = r * G + s;
            if (j >= n) continue;
            const double m = fabs(cr[j]) + fabs(ci[j]);
            if (!(fabs(ci[j]) < 1e-6 * m)) continue;
#pragma unroll 1
            for (int k = 0; k < n; k++) {
                if (k == j || !(fabs(ci[k]) < 1e-6 * m)) continue;
                if (fabs(cr[k] - cr[j]) < 1e-3 * m) { zim[r] += (j < k ? 1e-6 : -1e-6) * m; break; }
            }
        }
    }
    {
        int settled = 0;
        double prev = 1e300;
        bool done = !active;
        // Isolated roots (every one more than a tenth of its modulus from the
        // others, judged on the single-precision approximations): the
        // iteration converges cubically from ~1e-6, so one FP64 sweep whose
        // corrections are all below 1e-6 leaves them within rounding and no
        // confirming sweep is needed.
        bool iso = true;
#pragma unroll 1
        for (int it = 0; it < 200; it++) {
            double br[4], bi[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                br[k] = G == 1 ? zre[k / G] : __shfl_sync(full, zre[k / G], k % G, G);
                bi[k] = G == 1 ? zim[k / G] : __shfl_sync(full, zim[k / G], k % G, G);
            }
            if (it == 0) {
#pragma unroll 1
                for (int j = 0; j < n; j++) {
                    const float mj = sqrtf((float)(br[j] * br[j] + bi[j] * bi[j]));
#pragma unroll 1
                    for (int k = 0; k < n; k++) {
                        if (k == j) continue;
                        const float dr_ = (float)(br[j] - br[k]), di_ = (float)(bi[j] - bi[k]);
                        if (!(sqrtf(dr_ * dr_ + di_ * di_) > 0.1f * mj)) iso = false;
                    }
                }
            }
            double worst = 0.0;
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int j = r * G + s;
                if (done || j >= n) continue;
                cd zj = cmk(br[j], bi[j]), p, dp;
                horner(c, n, zj, p, dp);
                if (p.re == 0 && p.im == 0) continue;
                cd ratio = cmul(p, crcp(dp));
                cd sm = cmk(0, 0);
#pragma unroll 1
                for (int k = 0; k < n; k++)
                    if (k != j) sm = cadd(sm, crcp(csub(zj, cmk(br[k], bi[k]))));
                cd w = cmul(ratio, crcp(csub(cmk(1, 0), cmul(ratio, sm))));
                zj = csub(zj, w);
                zre[r] = zj.re; zim[r] = zj.im;
                const double rel = cnorm(w) * ddiv(1.0, cnorm(zj) + 1e-300);
                if (!(rel <= worst)) worst = rel;   // a NaN counts as the worst
            }
            if (G > 1) {
#pragma unroll
                for (int o = 1; o < G; o <<= 1) {
                    double v = __shfl_xor_sync(full, worst, o, G);
                    if (!(v <= worst)) worst = v;
                }
            }
            if (!done) {
                if (worst < 1e-30 || (it == 0 && iso && worst < 1e-12)) { if (++settled >= 1) done = true; }
                else if (it >= 4 && worst >= 0.25 * prev && worst < 1e-24) done = true;
                prev = worst;
            }
            if (__all_sync(full, done)) break;
        }
    }
    // A root whose imaginary part is negligible (|Im| <= 1e-12 |z|: the
    // classification's test) is put on the real axis.  Roots closer than a
    // tenth of their modulus to another root (near-multiple roots, as near
    // the no-Big-Bang boundary) are then polished by Newton steps on the
    // original coefficients (the monic ones carry the rounding of the
    // division by alpha_n), evaluated by the compensated scheme, each by the
    // lane that owns it; an isolated root is already within an ulp or two
    // after the sweeps (the rounding of the monic coefficients moves it by
    // its condition number, small when it is isolated), so it skips the
    // polish and its FP64 work.
    {
        double cr[4], ci[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            cr[k] = G == 1 ? zre[k / G] : __shfl_sync(full, zre[k / G], k % G, G);
            ci[k] = G == 1 ? zim[k / G] : __shfl_sync(full, zim[k / G], k % G, G);
        }
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int j = r * G + s;
            if (!active || j >= n) continue;
            cd zj = cmk(zre[r], zim[r]);
            const double mz = cabs_(zj);
            if (fabs(zj.im) <= 1e-12 * mz) zj.im = 0.0;
            bool isolated = true;
#pragma unroll 1
            for (int k = 0; k < n; k++)
                if (k != j && !(cabs_(csub(cmk(cr[k], ci[k]), cmk(cr[j], ci[j]))) > 0.1 * mz)) isolated = false;
            if (!isolated) polish_root(alpha, n, zj);
            zre[r] = zj.re; zim[r] = zj.im;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; k++)
        z[k] = G == 1 ? cmk(zre[k / G], zim[k / G])
                      : cmk(__shfl_sync(full, zre[k / G], k % G, G), __shfl_sync(full, zim[k / G], k % G, G));
}

// Record of one cosmology from its parameter row p[ncol] = (H0, Om, OL, Or[, Ok]);
// returns the status code.  Called by the G lanes of a group together (see
// group_roots); `active` is false for lanes past the last cosmology.
template <int G> __device__ int prep_one(const double* p, int ncol, double* rec, bool active) {
    double H0 = p[0], Om = p[1], OL = p[2], Or = p[3];
    double Ok = ncol >= 5 ? p[4] : 1.0 - Om - OL - Or;
    // the further components of fn4 (7-column rows): Os (w = -1/3) scales as
    // (1+z)^2 like curvature but stays out of the curvature map, Ox (w = -2/3)
    // as (1+z); with them every density is an independent direction
    const double Os = ncol >= 7 ? p[5] : 0.0, Ox = ncol >= 7 ? p[6] : 0.0;
    for (int i = 0; i < NREC; i++) rec[i] = 0;
    int st = ST_OK, kind = 0;
    const int K = ncol - 1;
    bool finite = isfinite(H0) && isfinite(Om) && isfinite(OL) && isfinite(Or) && isfinite(Ok) &&
                  isfinite(Os) && isfinite(Ox);
    int n = Or > 0 ? 4 : 3;
    if (!finite || !(H0 > 0) || Or < 0 || (n == 3 && !(Om > 0))) st = ST_INVALID;
    cd z[4];
    double alpha[5] = {OL, Ox, Ok + Os, Om, Or};
    double an = alpha[n];
    double c[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    c[n] = 1.0;
    if (st == ST_OK) {
        const double ian = ddiv(1.0, an);
        for (int k = 0; k <= n; k++) c[k] = alpha[k] * ian;
        c[n] = 1.0;
    }
    // A triple root at rho = 0 (x = 1 + z = 0): OL = Ox = Ok + Os = 0 to within
    // the rounding of the closure, so that E^2 = x^3 (Or x + Om) (flat matter +
    // radiation; Einstein-de Sitter when Or = 0).  The root iteration cannot
    // separate a triple root (its error would be of order eps^(1/3)), so the
    // roots are set exactly: rho = 0 three times and rho_A = -Om/Or.  The
    // reductions (3.7)-(3.9) / (B.1)-(B.3) then hold with the repeated roots
    // (the factors d_ij that vanish only multiply terms that drop out).  The
    // root derivatives of App. A are singular at a multiple root, so the
    // tangent slots of such a row are NaN (no gradient).
    const double dtol = 8.0 * 2.220446049250313e-16 * (fabs(Om) + fabs(Or) + fabs(OL) + fabs(Ok) + 1.0);
    const bool triple0 = st == ST_OK && fabs(OL) <= dtol && fabs(Ox) <= dtol && fabs(Ok + Os) <= dtol;
    group_roots<G>(c, alpha, n, active && st == ST_OK && !triple0, z);   // every lane, outside any divergent branch
    if (triple0) {
        z[0] = cmk(n == 4 ? -Om / Or : 0.0, 0.0);
        for (int i = 1; i < 4; i++) z[i] = cmk(0.0, 0.0);
    }
    if (st == ST_OK) {
        // classification: real when the imaginary part is negligible
        int nreal = 0, ir[4], ic[4], ncx = 0;
        #pragma unroll 1
        for (int i = 0; i < n; i++) {
            if (triple0 || fabs(z[i].im) <= 1e-12 * cabs_(z[i])) {   // (polished on the axis already)
                z[i].im = 0;
                ir[nreal++] = i;
            }
            else ic[ncx++] = i;
        }
        #pragma unroll 1
        for (int i = 0; i < nreal; i++)
            if (z[ir[i]].re >= 1.0) st = ST_NO_BIG_BANG;   // real root at z >= 0 (Sec. 3, Fig. 1)
        // order reals by decreasing |rho| (fn15: largest roots of E^2(z+1))
        #pragma unroll 1
        for (int i = 0; i < nreal; i++)
            for (int j = i + 1; j < nreal; j++)
                if (fabs(z[ir[j]].re) > fabs(z[ir[i]].re)) { int t = ir[i]; ir[i] = ir[j]; ir[j] = t; }
        cd A, Bv, P1, P2;
        bool cpair = false;
        if (n == 4 && nreal == 2 && ncx == 2) {
            kind = 0; A = z[ir[0]]; Bv = z[ir[1]]; cpair = true;
            P1 = z[ic[0]].im > 0 ? z[ic[0]] : z[ic[1]];
            P1.im = 0.5 * (fabs(z[ic[0]].im) + fabs(z[ic[1]].im));
            P1.re = 0.5 * (z[ic[0]].re + z[ic[1]].re);
        } else if (n == 4 && nreal == 4) {
            kind = 1; A = z[ir[0]]; Bv = z[ir[1]]; P1 = z[ir[2]]; P2 = z[ir[3]];
        } else if (n == 3 && nreal == 1 && ncx == 2) {
            kind = 2; A = z[ir[0]]; Bv = cmk(0, 0); cpair = true;
            P1 = z[ic[0]].im > 0 ? z[ic[0]] : z[ic[1]];
            P1.im = 0.5 * (fabs(z[ic[0]].im) + fabs(z[ic[1]].im));
            P1.re = 0.5 * (z[ic[0]].re + z[ic[1]].re);
        } else if (n == 3 && nreal == 3) {
            kind = 3; A = z[ir[0]]; Bv = cmk(0, 0); P1 = z[ir[1]]; P2 = z[ir[2]];
        } else if (st == ST_OK) {
            st = ST_UNSUPPORTED;   // e.g. two complex pairs (no real root)
        }
        if (st == ST_OK || st == ST_NO_BIG_BANG) {
            // roots in x = 1+z for the derivatives; stored in z
            cd rho[4];
            int nr = 0;
            rho[nr++] = A;
            if (n == 4) rho[nr++] = Bv;
            rho[nr++] = P1;
            rho[nr++] = cpair ? cmk(P1.re, -P1.im) : P2;
            if (A.re == 0.0 && !triple0) st = st == ST_OK ? ST_DEGENERATE : st;   // division by rho_A in eq. (3.8)
            rec[RF_A] = A.re - 1.0;
            rec[RF_B] = (n == 4 ? Bv.re : 1.0) - 1.0;
            if (cpair) { rec[RF_PRE] = P1.re - 1.0; rec[RF_PIM] = P1.im; }
            else { rec[RF_PRE] = P1.re - 1.0; rec[RF_PIM] = P2.re - 1.0; }
            rec[RF_YA] = sqrt(-rec[RF_A]);
            rec[RF_YB] = sqrt(-rec[RF_B]);
            if (cpair) { cd y = csqrt_(cmk(-rec[RF_PRE], -rec[RF_PIM])); rec[RF_YPRE] = y.re; rec[RF_YPIM] = y.im; }
            else { rec[RF_YPRE] = sqrt(-rec[RF_PRE]); rec[RF_YPIM] = sqrt(-rec[RF_PIM]); }
            // App. A (eqs. A.2-A.4): d rho_j / d c_i = -rho_j^i / prod_{m != j} (rho_j - rho_m).
            // Summed over the coefficients c_i = alpha_i / alpha_n of the monic
            // polynomial this is
            //   d rho_j / d theta_k = -(dE^2/dtheta_k)(rho_j) / (alpha_n prod_{m != j} (rho_j - rho_m)),
            // with dE^2/dOm = x^3, dE^2/dOL = 1, dE^2/dOr = x^4, dE^2/dOk = dE^2/dOs = x^2,
            // dE^2/dOx = x, and -x^2 added to the first three under the closure.
            // With G lanes per cosmology, lane j of the group takes root j and
            // the group exchanges the results (the G lanes of a group take the
            // same branches: one cosmology).
            cd dr[4][RF_KT];
            const int sg = G > 1 ? (int)(threadIdx.x & (G - 1)) : 0;
            int degen = 0;
            #pragma unroll 1
            for (int j = 0; j < nr; j++) {
                if (G > 1 && j != sg) continue;
                const cd x = rho[j], x2 = cmul(x, x);
                cd e2p = cmk(an, 0);
                #pragma unroll 1
                for (int m2 = 0; m2 < nr; m2++)
                    if (m2 != j) e2p = cmul(e2p, csub(x, rho[m2]));
                const bool degenerate = e2p.re == 0 && e2p.im == 0;
                if (degenerate) degen = 1;
                const cd inv = degenerate ? cmk(nan(""), nan("")) : crcp(e2p);
                const cd x3 = cmul(x2, x);
                const cd cx2 = ncol == 4 ? x2 : cmk(0, 0);
                #pragma unroll 1
                for (int k = 0; k < K; k++) {
                    const cd g = k == 0 ? csub(x3, cx2) : k == 1 ? csub(cmk(1, 0), cx2)
                               : k == 2 ? csub(cmul(x3, x), cx2) : k == 5 ? x : x2;
                    cd d = cmul(g, inv);
                    dr[j][k] = cmk(-d.re, -d.im);
                    if (n == 3 && k == 2) dr[j][k] = cmk(nan(""), nan(""));  // no Or direction in a cubic
                }
            }
            if (G > 1) {
                const unsigned gmask = ((1u << G) - 1) << ((threadIdx.x & 31) & ~(G - 1));
                #pragma unroll
                for (int o = 1; o < G; o <<= 1) degen |= __shfl_xor_sync(gmask, degen, o, G);
                #pragma unroll 1
                for (int j = 0; j < nr; j++)
                    #pragma unroll 1
                    for (int k = 0; k < K; k++) {
                        dr[j][k].re = __shfl_sync(gmask, dr[j][k].re, j, G);
                        dr[j][k].im = __shfl_sync(gmask, dr[j][k].im, j, G);
                    }
            }
            if (degen && !triple0) st = (st == ST_OK) ? ST_DEGENERATE : st;
            // big-root quantities of the quartic, scaled by lam = Or (see quartic_integrals)
            if (n == 4) {
                double rA = A.re;                  // rho_A
                rec[RF_LAM] = Or;
                rec[RF_AA] = -Or * (rA - 1.0);
                rec[RF_MA] = Or * rA;
                const double irA = ddiv(1.0, rA);
                rec[RF_EPSA] = -irA;
                rec[RF_RHOA] = rA;
                // Tangents of m_A = lam rho_A = y from the scaled quartic
                //   F(y) = y^4 + Om y^3 + (Ok + Os) Or y^2 + Ox Or^2 y + OL Or^3 = Or^3 E^2(rho_A) = 0,
                // dy = -(dF/dtheta) / (dF/dy), a ratio of O(1) terms: in the Or
                // direction rho_A d lam and lam d rho_A are each O(Om/Or) and cancel.
                // a_A = -lam (rho_A - 1) = -y + lam.
                const double y = Or * rA, Oks = Ok + Os;
                const double iFy = ddiv(1.0, y * y * (4.0 * y + 3.0 * Om) + 2.0 * Oks * Or * y + Ox * Or * Or);
                const double cl = ncol == 4 ? 1.0 : 0.0, FOk = Or * y * y;
                const double Fth[RF_KT] = {y * y * y - cl * FOk, Or * Or * Or - cl * FOk,
                                           Oks * y * y + 2.0 * Ox * Or * y + 3.0 * OL * Or * Or - cl * FOk, FOk, FOk,
                                           Or * Or * y};
                #pragma unroll 1
                for (int k = 0; k < K; k++) {
                    double dl = (k == 2) ? 1.0 : 0.0, dA = dr[0][k].re;
                    const double dy = -Fth[k] * iFy;
                    rec[RF_DLAM + k] = dl;
                    rec[RF_DAA + k] = dl - dy;
                    rec[RF_DMA + k] = dy;
                    rec[RF_DEPSA + k] = dA * (irA * irA);
                    rec[RF_DRHOA + k] = dA;
                }
            }
            // q_j = -1/r_j (dq_j = dr_j / r_j^2) for the normalised Carlson arguments
            {
                double rA = A.re - 1.0;
                const double iA = rA != 0.0 ? ddiv(1.0, rA) : 0.0;
                rec[RF_QA] = -iA;
                for (int k = 0; k < K; k++) rec[RF_DQA + k] = dr[0][k].re * (iA * iA);
                if (n == 4) {
                    double rB = Bv.re - 1.0;
                    const double iB = rB != 0.0 ? ddiv(1.0, rB) : 0.0;
                    rec[RF_QB] = -iB;
                    for (int k = 0; k < K; k++) rec[RF_DQB + k] = dr[1][k].re * (iB * iB);
                }
                const int jq = n == 4 ? 2 : 1;
                if (cpair) {
                    cd r = cmk(P1.re - 1.0, P1.im);
                    cd q = cdiv(cmk(-1.0, 0.0), r);
                    rec[RF_QPRE] = q.re;
                    rec[RF_QPIM] = q.im;
                    const cd q2 = cmul(q, q);   // dq = dr / r^2 = q^2 dr
                    for (int k = 0; k < K; k++) {
                        cd dq = cmul(dr[jq][k], q2);
                        rec[RF_DQPRE + k] = dq.re;
                        rec[RF_DQPIM + k] = dq.im;
                    }
                } else {
                    double r1 = P1.re - 1.0, r2 = P2.re - 1.0;
                    const double i1 = r1 != 0.0 ? ddiv(1.0, r1) : 0.0, i2 = r2 != 0.0 ? ddiv(1.0, r2) : 0.0;
                    rec[RF_QPRE] = -i1;
                    rec[RF_QPIM] = -i2;
                    for (int k = 0; k < K; k++) {
                        rec[RF_DQPRE + k] = dr[jq][k].re * (i1 * i1);
                        rec[RF_DQPIM + k] = dr[jq + 1][k].re * (i2 * i2);
                    }
                }
            }
            #pragma unroll 1
            for (int k = 0; k < K; k++) {
                rec[RF_DA + k] = dr[0][k].re;
                rec[RF_DB + k] = n == 4 ? dr[1][k].re : 0.0;
                int jp = n == 4 ? 2 : 1;
                if (cpair) { rec[RF_DPRE + k] = dr[jp][k].re; rec[RF_DPIM + k] = dr[jp][k].im; }
                else { rec[RF_DPRE + k] = dr[jp][k].re; rec[RF_DPIM + k] = dr[jp + 1][k].re; }
            }
        }
    }
    // prefactors: alpha_m^-1/2 (Or for the quartic, Om for the cubic, eq. 3.2 / fn13)
    double amh = ddiv(1.0, sqrt(n == 4 ? Or : Om));
    rec[RF_AMH] = amh;
    rec[RF_OK] = Ok;
    rec[RF_H0] = H0;
    const double iH0 = ddiv(1.0, H0);
    rec[RF_DH] = LCDM_C_KMS * iH0;
    rec[RF_TH] = LCDM_HUBBLE_GYR * iH0;
    rec[RF_KIND] = kind;
    // N = sqrt(E^2(0) / alpha_n): E^2(0) = Om + OL + Or + Ok (+ Os + Ox), exactly 1 under the closure
    const double S0 = ncol == 4 ? 1.0 : Om + OL + Or + Ok + Os + Ox;
    const double iOm = ddiv(1.0, Om);
    const double nrm = n == 4 ? sqrt(S0) : sqrt(S0 * iOm);
    const double inrm = ddiv(1.0, nrm);
    rec[RF_NRM] = nrm;
    #pragma unroll 1
    for (int k = 0; k < K; k++) {
        const double dS = ncol == 4 ? 0.0 : 1.0, dOm = k == 0 ? 1.0 : 0.0;
        rec[RF_DNRM + k] = n == 4 ? 0.5 * dS * inrm : 0.5 * (dS * Om - S0 * dOm) * inrm * (iOm * iOm);
        if (n == 3 && k == 2) rec[RF_DNRM + k] = nan("");
    }
    #pragma unroll 1
    for (int k = 0; k < K; k++) {
        rec[RF_DAMH + k] = 0;
        if (n == 4 && k == 2) rec[RF_DAMH + k] = -0.5 * amh * amh * amh;
        if (n == 3 && k == 0) rec[RF_DAMH + k] = -0.5 * amh * amh * amh;
        if (n == 3 && k == 2) rec[RF_DAMH + k] = nan("");
        rec[RF_DOK + k] = ncol == 4 ? -1.0 : (k == 3 ? 1.0 : 0.0);
    }
    return st;
}

// G lanes per cosmology (see group_roots); grad / loglike (optional): rows
// initialised to 0 (NaN for a bad status).  Launched with 32-thread blocks
// over G B threads.
template <int G>
__global__ void prep_kernel(const double* __restrict__ params, int64_t B, int ncol, double* __restrict__ recD,
                            float2* __restrict__ recF, int32_t* __restrict__ status, double* __restrict__ grad,
                            double* __restrict__ loglike) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t b = t / G;
    const int j = (int)(t % G);
    const bool inb = b < B;
    // lanes past the end work on a copy of the last row and write nothing
    const double* prow = params + (inb ? b : B - 1) * ncol;
    double rec[NREC];
    const int st = prep_one<G>(prow, ncol, rec, inb);
    if (!inb) return;
    double* rd = recD + b * NREC;
    float2* rf = recF + b * NREC;
    #pragma unroll 1
    for (int i = j; i < NREC; i += G) {
        rd[i] = rec[i];
        float h = (float)rec[i];
        rf[i] = make_float2(h, (float)(rec[i] - (double)h));
    }
    if (j != 0) return;
    status[b] = st;
    double init = st == ST_OK ? 0.0 : nan("");
    if (grad)
        for (int k = 0; k < ncol; k++) grad[b * ncol + k] = init;
    if (loglike) loglike[b] = init;
}

}  // namespace lcdm
