/*
 * lcdm_oracle.c -- plain FP64 CPU oracle for LambdaCDM+radiation+curvature
 * distances (Karchev, "Analytic auto-differentiable LambdaCDM cosmography").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA path and never calls it.
 *
 * Contents (each function cites the passage it follows):
 *   O1  oracle_quad_distances : adaptive Gauss-Legendre quadrature of the
 *       defining integrals (2.3)-(2.5), written in the scale factor a.
 *   O4  (same call, jac != NULL): Leibniz-rule gradients of the same
 *       integrals with respect to the density parameters (fn23 of the paper
 *       describes this approach), plus the curvature / modulus chain rule.
 *   O2  oracle_carlson_distances : eqs. (3.7)-(3.9) (quartic) and
 *       (B.1)-(B.3) (cubic) assembled in complex FP64 from given roots.
 *   Carlson R_F, R_J, R_C, R_D (eqs. 2.6-2.9) by Carlson's duplication
 *       algorithm (the paper's ref. [10]), complex arguments, with Cauchy
 *       principal values for negative real w (R_J) and y (R_C) (Sec. 2.2).
 *
 * Everything is written for clarity, not speed: no blocking, no fusion.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* Physical constants (standard values, stated here independently). */
#define C_KMS 299792.458                 /* speed of light, km/s            */
#define HUBBLE_TIME_GYR 977.7922216807891 /* (1 Mpc / 1 km) / (1 Gyr / 1 s)  */
/* 1 Mpc = 3.0856775814913673e19 km; 1 Gyr = 1e9 Julian years of 365.25 d.  */

/* ------------------------------------------------------------------------ */
/* Deliberate-mistake switch.  Tests set a non-zero value to check that the  */
/* pins catch a plausible error; 0 (default) is the correct oracle.          */
/*   1: drop the E3/14 term of the R_F series                                */
/*   2: flip the sign of the R_C term in eq. (3.8)                           */
/*   3: transpose X_i <-> Y_i in u_ij (quartic and cubic)                    */
/*   4: drop the (1+z) factor of the luminosity distance                     */
/*   5: drop the -a^2 closure term from the Omega_m Leibniz gradient          */
/*   6: replace R_C(1, 1+e_m) by 1 in the duplication sum of R_J            */
/*   7: use sqrt(-r) for Y_m = sqrt(z1 - r_m) (forget the lower limit)      */
/*   8: drop the R_C term of the z2 -> infinity limit of eq. (3.8)          */
/* ------------------------------------------------------------------------ */
static int g_mutation = 0;
void oracle_set_mutation(int m) { g_mutation = m; }

/* ======================================================================== */
/* Carlson symmetric integrals by duplication (ref. [10]).                  */
/* Tolerance r: the series is truncated once every normalised deviation is  */
/* below the level at which the neglected terms are smaller than r.         */
/* ======================================================================== */
#define CARLSON_R 1e-17
#define CARLSON_MAXIT 200

static double maxabs3(cplx a, cplx b, cplx c) {
    double m = cabs(a);
    if (cabs(b) > m) m = cabs(b);
    if (cabs(c) > m) m = cabs(c);
    return m;
}

/* R_C(x, y) = R_F(x, y, y), eq. (2.8). */
static cplx rc_dup(cplx x, cplx y) {
    cplx A0 = (x + 2.0 * y) / 3.0, A = A0;
    double Q = pow(3.0 * CARLSON_R, -1.0 / 8.0) * cabs(A0 - x);
    double f = 1.0; /* 4^-m */
    int m = 0;
    while (f * Q >= cabs(A) && m < CARLSON_MAXIT) {
        cplx lam = 2.0 * csqrt(x) * csqrt(y) + y;
        A = (A + lam) / 4.0; x = (x + lam) / 4.0; y = (y + lam) / 4.0;
        f /= 4.0; m++;
    }
    cplx s = (y - A) / A; /* deviation of y from the running mean */
    cplx series = 1.0 + s * s * (3.0 / 10.0 + s * (1.0 / 7.0 + s * (3.0 / 8.0 + s * (9.0 / 22.0
                  + s * (159.0 / 208.0 + s * (9.0 / 8.0))))));
    return series / csqrt(A);
}

cplx oracle_rc(cplx x, cplx y) {
    /* Cauchy principal value for real negative y (Sec. 2.2): the pole of the
     * integrand is moved off the path with R_C(x,-q) = sqrt(x/(x+q)) R_C(x+q, q). */
    if (cimag(y) == 0.0 && creal(y) < 0.0 && cimag(x) == 0.0 && creal(x) >= 0.0) {
        double q = -creal(y);
        return csqrt(x / (x + q)) * rc_dup(x + q, q);
    }
    return rc_dup(x, y);
}

/* R_F(x, y, z), eq. (2.6). */
cplx oracle_rf(cplx x, cplx y, cplx z) {
    cplx x0 = x, y0 = y, A0 = (x + y + z) / 3.0, A = A0;
    double Q = pow(3.0 * CARLSON_R, -1.0 / 6.0) * maxabs3(A0 - x, A0 - y, A0 - z);
    double f = 1.0;
    int m = 0;
    while (f * Q >= cabs(A) && m < CARLSON_MAXIT) {
        cplx sx = csqrt(x), sy = csqrt(y), sz = csqrt(z);
        cplx lam = sx * sy + sx * sz + sy * sz;
        A = (A + lam) / 4.0; x = (x + lam) / 4.0; y = (y + lam) / 4.0; z = (z + lam) / 4.0;
        f /= 4.0; m++;
    }
    cplx X = f * (A0 - x0) / A, Y = f * (A0 - y0) / A, Z = -(X + Y);
    cplx E2 = X * Y - Z * Z, E3 = X * Y * Z;
    cplx series = 1.0 - E2 / 10.0 + (g_mutation == 1 ? 0.0 : E3 / 14.0) + E2 * E2 / 24.0
                  - 3.0 * E2 * E3 / 44.0;
    return series / csqrt(A);
}

/* R_J(x, y, z, p) for p not on the negative real axis, eq. (2.7). */
static cplx rj_dup(cplx x, cplx y, cplx z, cplx p) {
    cplx x0 = x, y0 = y, z0 = z, A0 = (x + y + z + 2.0 * p) / 5.0, A = A0;
    cplx delta = (p - x) * (p - y) * (p - z);
    double Q = maxabs3(A0 - x, A0 - y, A0 - z);
    if (cabs(A0 - p) > Q) Q = cabs(A0 - p);
    Q *= pow(CARLSON_R / 4.0, -1.0 / 6.0);
    double f = 1.0;
    cplx sum = 0.0;
    int m = 0;
    while (f * Q >= cabs(A) && m < CARLSON_MAXIT) {
        cplx sx = csqrt(x), sy = csqrt(y), sz = csqrt(z), sp = csqrt(p);
        cplx lam = sx * sy + sx * sz + sy * sz;
        cplx d = (sp + sx) * (sp + sy) * (sp + sz);
        cplx e = f * f * f * delta / (d * d);
        if (g_mutation == 6)
            sum += f / d;
        else
            sum += f * rc_dup(1.0, 1.0 + e) / d;
        A = (A + lam) / 4.0; x = (x + lam) / 4.0; y = (y + lam) / 4.0; z = (z + lam) / 4.0;
        p = (p + lam) / 4.0;
        f /= 4.0; m++;
    }
    cplx X = f * (A0 - x0) / A, Y = f * (A0 - y0) / A, Z = f * (A0 - z0) / A;
    cplx P = -(X + Y + Z) / 2.0;
    cplx E2 = X * Y + X * Z + Y * Z - 3.0 * P * P;
    cplx E3 = X * Y * Z + 2.0 * E2 * P + 4.0 * P * P * P;
    cplx E4 = (2.0 * X * Y * Z + E2 * P + 3.0 * P * P * P) * P;
    cplx E5 = X * Y * Z * P * P;
    cplx series = 1.0 - 3.0 * E2 / 14.0 + E3 / 6.0 + 9.0 * E2 * E2 / 88.0 - 3.0 * E4 / 22.0
                  - 9.0 * E2 * E3 / 52.0 + 3.0 * E5 / 26.0;
    return f * series / (A * csqrt(A)) + 6.0 * sum;
}

static int is_real(cplx v) { return cimag(v) == 0.0; }

/* R_J with the Cauchy principal value for real negative p (Sec. 2.2).
 * The triple must then be real-valued as a set (three reals, or one real and
 * a conjugate pair); the real member goes to the third slot and
 *   (q+z) R_J(x,y,z,-q) = (s-z) R_J(x,y,z,s) - 3 R_F(x,y,z)
 *                         + 3 sqrt(xyz/(xy+sq)) R_C(xy+sq, sq),
 *   s = (z(x+y+q) - xy)/(z+q),
 * which is only used when s > 0 (otherwise NaN is returned). */
cplx oracle_rj(cplx x, cplx y, cplx z, cplx p) {
    if (!(is_real(p) && creal(p) < 0.0)) return rj_dup(x, y, z, p);
    cplx v[3] = {x, y, z};
    int ir = -1;
    for (int i = 0; i < 3; i++)
        if (is_real(v[i]) && (ir < 0 || creal(v[i]) > creal(v[ir]))) ir = i;
    if (ir < 0) return NAN;
    cplx zz = v[ir], xx = v[(ir + 1) % 3], yy = v[(ir + 2) % 3];
    double q = -creal(p);
    cplx s = (zz * (xx + yy + q) - xx * yy) / (zz + q);
    if (!(creal(s) > 0.0)) return NAN;
    cplx xy = xx * yy;
    cplx val = (s - zz) * rj_dup(xx, yy, zz, s) - 3.0 * oracle_rf(xx, yy, zz)
               + 3.0 * csqrt(xx * yy * zz / (xy + s * q)) * oracle_rc(xy + s * q, s * q);
    return val / (q + zz);
}

/* R_D(x, y, z) = R_J(x, y, z, z), eq. (2.9). */
cplx oracle_rd(cplx x, cplx y, cplx z) { return rj_dup(x, y, z, z); }

/* Batch entry for tests: kind 0=R_F 1=R_J 2=R_C 3=R_D; args [n][4] complex as
 * (re,im) pairs; out [n] complex as (re,im). */
void oracle_carlson_batch(int kind, int64_t n, const double* args, double* out) {
    for (int64_t i = 0; i < n; i++) {
        const double* a = args + 8 * i;
        cplx x = a[0] + I * a[1], y = a[2] + I * a[3], z = a[4] + I * a[5], p = a[6] + I * a[7];
        cplx r = 0;
        switch (kind) {
            case 0: r = oracle_rf(x, y, z); break;
            case 1: r = oracle_rj(x, y, z, p); break;
            case 2: r = oracle_rc(x, y); break;
            case 3: r = oracle_rd(x, y, z); break;
            default: r = NAN;
        }
        out[2 * i] = creal(r);
        out[2 * i + 1] = cimag(r);
    }
}

/* ======================================================================== */
/* Curvature map and observables (Sec. 2.1.1; ref. [59] eqs. 13.47, 13.57;  */
/* distance modulus fn22).                                                  */
/* ======================================================================== */

/* S_k(D) for dimensionless comoving distance D and curvature Ok, together
 * with dS/dD and dS/dOk. */
static void curv_map(double D, double Ok, double* S, double* SD, double* Sk) {
    double u = Ok * D * D;
    if (fabs(u) < 1e-2) {
        /* Taylor series in u = Ok D^2 (exact to double precision here). */
        double s = 0, sd = 0, sk = 0, term = 1.0, fact = 1.0;
        for (int n = 0; n < 9; n++) {
            /* S = D sum u^n/(2n+1)!, S_D = sum u^n/(2n)!, S_k = D^3 sum n u^(n-1)/(2n+1)! */
            double f2n1 = fact * (2 * n + 1);      /* (2n+1)! */
            s += D * term / f2n1;
            sd += term / fact;                     /* fact = (2n)! */
            if (n > 0) sk += D * D * D * n * (term / u) / f2n1;
            term *= u;
            fact *= (2 * n + 1) * (2 * n + 2);
        }
        if (u == 0.0) sk = D * D * D / 6.0;
        *S = s; *SD = sd; *Sk = sk;
        return;
    }
    if (Ok > 0) {
        double r = sqrt(Ok);
        *S = sinh(r * D) / r;
        *SD = cosh(r * D);
    } else {
        double r = sqrt(-Ok);
        *S = sin(r * D) / r;
        *SD = cos(r * D);
    }
    *Sk = (D * (*SD) - *S) / (2.0 * Ok);
}

/* ======================================================================== */
/* O1 / O4: adaptive Gauss-Legendre quadrature in the scale factor.         */
/*   chi = (c/H0) int_a^1 da / sqrt(Q(a)),                                  */
/*   t   = (1/H0) int_a^1 a da / sqrt(Q(a)),                                */
/*   X   = (c/H0) int_a^1 a^-2 da / sqrt(Q(a)),                             */
/* with Q(a) = Or + Om a + Ok a^2 + OL a^4 = a^4 E^2(z), a = 1/(1+z); this  */
/* is eqs. (2.3)-(2.5) after dz = -da/a^2.                                  */
/* ======================================================================== */
#define NGL 15
static double gl_x[NGL], gl_w[NGL];
static int gl_ready = 0;

static void gl_init(void) {
    /* Gauss-Legendre nodes: Newton iteration on the Legendre polynomial P_n. */
    const int n = NGL;
    for (int i = 0; i < n; i++) {
        double x = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-17) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; k++) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1; p1 = p2;
        }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    gl_ready = 1;
}

#define NCOMP 18 /* 3 forward integrands + 3 weights x 5 coefficient functions */

/* Density parameters; Os (w = -1/3, scaling as (1+z)^2 like curvature but
 * outside the curvature map) and Ox (w = -2/3, scaling as (1+z)) are the
 * other components the method allows (fn4); both 0 unless given. */
typedef struct { double Om, OL, Or, Ok, Os, Ox; } cosmo_t;

/* Integrand vector at scale factor a.
 * [0..2]: w(a)/sqrt(Q) for w = 1, a, a^-2.
 * [3 + 5*iw + ig]: -(1/2) w(a) g(a) Q^-3/2 for g = dQ/dOm = a, dQ/dOL = a^4,
 *                  dQ/dOr = 1, dQ/dOk = dQ/dOs = a^2, dQ/dOx = a^3 (Leibniz
 *                  rule under the integral). */
/* Q(a) by Horner's rule with the rounding error of each step carried along
 * exactly (error-free sum and product; the compensated Horner scheme of
 * Graillat, Langlois and Louvet): near the deep minimum of Q at the
 * no-Big-Bang boundary (Fig. 1) its O(1) terms cancel to the small minimum
 * value, and a plain evaluation would leave the integrand with a relative
 * error of eps times their ratio. */
static double q_of_a(const cosmo_t* c, double a) {
    const double co[5] = {c->OL, c->Ox, c->Ok + c->Os, c->Om, c->Or};   /* highest power first */
    double h = co[0], err = 0.0;
    for (int k = 1; k < 5; k++) {
        double p = h * a, ep = fma(h, a, -p);
        double s = p + co[k], bb = s - p, es = (p - (s - bb)) + (co[k] - bb);
        err = err * a + (ep + es);
        h = s;
    }
    return h + err;
}

static void integrand(double a, const cosmo_t* c, double* out) {
    double Q = q_of_a(c, a);
    double iq = 1.0 / sqrt(Q), iq3 = iq / Q;
    double w[3] = {1.0, a, 1.0 / (a * a)};
    double g[5] = {a, a * a * a * a, 1.0, a * a, a * a * a};
    for (int iw = 0; iw < 3; iw++) {
        out[iw] = w[iw] * iq;
        for (int ig = 0; ig < 5; ig++) out[3 + 5 * iw + ig] = -0.5 * w[iw] * g[ig] * iq3;
    }
}

/* 15-point rule on [lo, hi] of the variable t.  The scale factor is
 *   mode 0: a = t;
 *   mode 1: a = anchor - t, next to the upper end a = anchor of the range, so
 *           that the width of a short interval, (z2 - z1)/((1+z1)(1+z2)), is
 *           exact;
 *   mode 2: a = t^2 with da = 2t dt, down to a = 0 (the z2 -> infinity limit,
 *           where the radiationless integrands grow like a^-1/2). */
static void gl_rule(const cosmo_t* c, int mode, double anchor, double lo, double hi, double* res,
                    double* absres) {
    double h = 0.5 * (hi - lo), mid = 0.5 * (hi + lo), v[NCOMP];
    for (int k = 0; k < NCOMP; k++) { res[k] = 0; if (absres) absres[k] = 0; }
    for (int i = 0; i < NGL; i++) {
        double tt = mid + h * gl_x[i];
        double a = mode == 0 ? tt : (mode == 1 ? anchor - tt : tt * tt);
        double wt = mode == 2 ? 2.0 * tt : 1.0;
        integrand(a, c, v);
        for (int k = 0; k < NCOMP; k++) {
            res[k] += gl_w[i] * h * wt * v[k];
            if (absres) absres[k] += gl_w[i] * h * wt * fabs(v[k]);
        }
    }
}

/* Adaptive bisection: an interval is accepted when, for every component,
 * the 15-point rule on it and the sum over its two halves agree to rtol times
 * the interval's own integral of |f| (so the total relative error is at most
 * about rtol).  At most MAX_INTERVALS intervals are evaluated; the return
 * value is the number of accepted intervals, negative if the cap was hit. */
#define MAX_INTERVALS 200000
#define KMASK_ALL 0x3ffff
/* the values and the four density directions of the standard components */
#define KMASK_STD (0x7 | (0xf << 3) | (0xf << 8) | (0xf << 13))
/* everything but the absorption distance and its derivatives (which diverge
 * as z2 -> infinity) */
#define KMASK_NO_X (KMASK_ALL & ~((1 << 2) | (0x1f << 13)))
/* components that decide the subdivision: the extra components' directions
 * only when they are parameters */
static int kmask_for(int ncol) { return ncol >= 7 ? KMASK_ALL : KMASK_STD; }
static int adapt(const cosmo_t* c, int mode, double anchor, double lo, double hi, double rtol, int kmask,
                 double* total) {
    double whole[NCOMP], wabs[NCOMP];
    gl_rule(c, mode, anchor, lo, hi, whole, wabs);
    for (int k = 0; k < NCOMP; k++) total[k] = 0;
    static double stk_lo[256], stk_hi[256], stk_v[256][NCOMP];
    int sp = 0, nacc = 0, nev = 0, capped = 0;
    stk_lo[0] = lo; stk_hi[0] = hi;
    memcpy(stk_v[0], whole, sizeof(whole));
    sp = 1;
    while (sp > 0) {
        sp--;
        double a = stk_lo[sp], b = stk_hi[sp], m = 0.5 * (a + b);
        double I1[NCOMP], L[NCOMP], R[NCOMP], La[NCOMP], Ra[NCOMP];
        memcpy(I1, stk_v[sp], sizeof(I1));
        gl_rule(c, mode, anchor, a, m, L, La);
        gl_rule(c, mode, anchor, m, b, R, Ra);
        nev++;
        int ok = 1;
        for (int k = 0; k < NCOMP; k++) {
            if (!(kmask >> k & 1)) continue;
            double err = fabs(L[k] + R[k] - I1[k]);
            if (err > rtol * (La[k] + Ra[k]) && err > 1e-300) { ok = 0; break; }
        }
        if (nev > MAX_INTERVALS) capped = 1;
        if (ok || capped || sp >= 250 || (b - a) < 1e-15 * (hi - lo)) {
            for (int k = 0; k < NCOMP; k++) total[k] += L[k] + R[k];
            nacc++;
        } else {
            stk_lo[sp] = m; stk_hi[sp] = b; memcpy(stk_v[sp], R, sizeof(R)); sp++;
            stk_lo[sp] = a; stk_hi[sp] = m; memcpy(stk_v[sp], L, sizeof(L)); sp++;
        }
    }
    return capped ? -nacc : nacc;
}

/* Breakpoints for the quadrature: near the no-Big-Bang boundary (Sec. 3,
 * Fig. 1) Q(a) has a deep minimum on the path and 1/sqrt(Q) a narrow peak,
 * which a coarse rule can step over.  The stationary points of Q in (lo, hi)
 * (roots of Q'(a) = Om + 2 Ok a + 4 OL a^3, found by bracketing on a grid and
 * bisection) and points at 1, 4, 16 and 64 peak widths sqrt(Q/|Q''|) on either
 * side become interval ends, in addition to 8 equal pieces. */
static int quad_breakpoints(const cosmo_t* c, double lo, double hi, double* bp) {
    int n = 0;
    const int NG = 256;
    double prev = 0, aprev = lo;
    for (int i = 0; i <= NG; i++) {
        double a = lo + (hi - lo) * i / NG;
        double d = c->Om + 2.0 * (c->Ok + c->Os) * a + 3.0 * c->Ox * a * a + 4.0 * c->OL * a * a * a;
        if (i > 0 && ((prev < 0) != (d < 0))) {
            double x0 = aprev, x1 = a, d0 = prev;
            for (int it = 0; it < 200; it++) {
                double xm = 0.5 * (x0 + x1);
                double dm = c->Om + 2.0 * (c->Ok + c->Os) * xm + 3.0 * c->Ox * xm * xm + 4.0 * c->OL * xm * xm * xm;
                if ((dm < 0) == (d0 < 0)) { x0 = xm; d0 = dm; } else x1 = xm;
            }
            double as = 0.5 * (x0 + x1);
            double Q = c->Or + c->Om * as + (c->Ok + c->Os) * as * as + c->Ox * as * as * as
                       + c->OL * as * as * as * as;
            double Q2 = 2.0 * (c->Ok + c->Os) + 6.0 * c->Ox * as + 12.0 * c->OL * as * as;
            double wd = (Q > 0 && Q2 != 0) ? sqrt(Q / fabs(Q2)) : 0.0;
            bp[n++] = as;
            for (int k = 1; k <= 64 && wd > 0; k *= 4) { bp[n++] = as - k * wd; bp[n++] = as + k * wd; }
        }
        prev = d; aprev = a;
    }
    for (int i = 1; i < 8; i++) bp[n++] = lo + (hi - lo) * i / 8.0;
    /* keep those inside, sorted */
    int m = 0;
    for (int i = 0; i < n; i++) if (bp[i] > lo && bp[i] < hi) bp[m++] = bp[i];
    for (int i = 1; i < m; i++) for (int j = i; j > 0 && bp[j - 1] > bp[j]; j--) { double t = bp[j]; bp[j] = bp[j - 1]; bp[j - 1] = t; }
    return m;
}

/* Adaptive quadrature over [lo, hi] of t (mode and anchor as in gl_rule),
 * split at the breakpoints (mapped to t); results added to total. */
static void integrate_pieces(const cosmo_t* c, int mode, double anchor, double lo, double hi, double rtol,
                             int kmask, double* total) {
    double bp[64], part[NCOMP];
    double alo = mode == 0 ? lo : (mode == 1 ? anchor - hi : lo * lo);
    double ahi = mode == 0 ? hi : (mode == 1 ? anchor - lo : hi * hi);
    int m = quad_breakpoints(c, alo, ahi, bp);
    double t[66];
    int nt = 0;
    t[nt++] = lo;
    for (int i = 0; i < m; i++) {
        double v = mode == 0 ? bp[i] : (mode == 1 ? anchor - bp[m - 1 - i] : sqrt(bp[i]));
        if (v > t[nt - 1] && v < hi) t[nt++] = v;
    }
    t[nt++] = hi;
    for (int i = 0; i + 1 < nt; i++) {
        adapt(c, mode, anchor, t[i], t[i + 1], rtol, kmask, part);
        for (int k = 0; k < NCOMP; k++) total[k] += part[k];
    }
}

/* The NCOMP integrals over z in [z1, z2] (z2 may be +infinity), i.e. over
 * a in [a2, a1] with a = 1/(1+z).  Next to a1 the variable is s = a1 - a over
 * [0, min(w, a1/2)], w = a1 - a2 = (z2 - z1)/((1+z1)(1+z2)) formed without
 * cancellation; the rest, [a2, a1/2], is integrated in a itself (in sqrt(a)
 * when a2 = 0).  Each part is further split at the breakpoints of
 * quad_breakpoints. */
static void integrate_between(const cosmo_t* c, double z1, double z2, double rtol, int kmask, double* Iv) {
    const int inf = isinf(z2);
    const double a1 = 1.0 / (1.0 + z1);
    const double w = inf ? a1 : (z2 - z1) / ((1.0 + z1) * (1.0 + z2));
    double I2[NCOMP];
    for (int k = 0; k < NCOMP; k++) Iv[k] = 0.0;
    integrate_pieces(c, 1, a1, 0.0, w < 0.5 * a1 ? w : 0.5 * a1, rtol, kmask, Iv);
    if (w > 0.5 * a1) {
        for (int k = 0; k < NCOMP; k++) I2[k] = 0.0;
        if (inf)
            integrate_pieces(c, 2, 0.0, 0.0, sqrt(0.5 * a1), rtol, kmask, I2);
        else
            integrate_pieces(c, 0, 0.0, 1.0 / (1.0 + z2), 0.5 * a1, rtol, kmask, I2);
        for (int k = 0; k < NCOMP; k++) Iv[k] += I2[k];
    }
}

/* params rows: (H0, Om, OL, Or) with the closure Ok = 1 - Om - OL - Or;
 * (H0, Om, OL, Or, Ok); or (H0, Om, OL, Or, Ok, Os, Ox) with the two further
 * components of fn4 (every density explicit). */
static void unpack_params(const double* p, int ncol, double* H0, cosmo_t* c) {
    *H0 = p[0];
    c->Om = p[1]; c->OL = p[2]; c->Or = p[3];
    c->Ok = (ncol >= 5) ? p[4] : 1.0 - p[1] - p[2] - p[3];
    c->Os = (ncol >= 7) ? p[5] : 0.0;
    c->Ox = (ncol >= 7) ? p[6] : 0.0;
}

/* Row of pair j in a CSR batch (offsets == NULL: every row holds nnz/B). */
static int64_t row_of(const int64_t* offsets, int64_t B, int64_t nnz, int64_t j) {
    if (!offsets) return j / (nnz / B);
    int64_t lo = 0, hi = B; /* offsets[lo] <= j < offsets[hi] */
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) / 2;
        if (offsets[mid] <= j) lo = mid; else hi = mid;
    }
    return lo;
}

/* O1 (+ O4) for one pair of limits z1 <= z2 (z2 finite), cosmology c:
 * o[6] = (chi, t, d_abs, d_M, d_L, mu) of eqs. (2.3)-(2.5) and Sec. 2.1.1;
 * J[6][ncol] (may be NULL) their derivatives w.r.t. the parameter columns.
 * d_M is the transverse comoving distance S_k(chi) between the two
 * redshifts; d_L = (1+z2) d_M / (1+z1)^2 is the luminosity distance of a
 * source at z2 seen by a comoving observer at z1 (the source's redshift
 * relative to that observer is (1+z2)/(1+z1) - 1; with z1 = 0 this is the
 * usual (1+z) d_M). */
static void quad_pair(const cosmo_t* c, double H0, int ncol, double z1, double z2, double rtol, double* o,
                      double* J) {
    double DH = C_KMS / H0, tH = HUBBLE_TIME_GYR / H0;
    double Iv[NCOMP];
    if (z2 == z1) {
        for (int k = 0; k < NCOMP; k++) Iv[k] = 0.0;
    } else {
        integrate_between(c, z1, z2, rtol, kmask_for(ncol), Iv);
    }
    double S, SD, Sk;
    curv_map(Iv[0], c->Ok, &S, &SD, &Sk);
    double lf = (g_mutation == 4 ? 1.0 : 1.0 + z2) / ((1.0 + z1) * (1.0 + z1));
    double dC = DH * Iv[0], t = tH * Iv[1], X = DH * Iv[2], dM = DH * S;
    double dL = lf * dM;
    double mu = 5.0 * log10(dL) + 25.0;
    o[0] = dC; o[1] = t; o[2] = X; o[3] = dM; o[4] = dL; o[5] = mu;
    if (!J) return;
    /* H0: every distance and time scales as 1/H0. */
    for (int k = 0; k < 5; k++) J[k * ncol + 0] = -o[k] / H0;
    J[5 * ncol + 0] = -5.0 / (log(10.0) * H0);
    /* Omega directions: dI_w/dtheta = sum_g (dQ/dtheta)_g-coefficients x J_w[g]. */
    for (int ip = 1; ip < ncol; ip++) {
        /* coefficients of (a, a^4, 1, a^2, a^3) in dQ/dtheta, and dOk/dtheta */
        double cg[5] = {0, 0, 0, 0, 0}, dOk = 0;
        if (ip == 1) cg[0] = 1;
        if (ip == 2) cg[1] = 1;
        if (ip == 3) cg[2] = 1;
        if (ip == 4 || ip == 5) cg[3] = 1;   /* Ok and Os enter Q alike */
        if (ip == 6) cg[4] = 1;
        if (ncol == 4) { /* closure: Ok = 1 - Om - OL - Or */
            if (!(g_mutation == 5 && ip == 1)) cg[3] = -1;
            dOk = -1;
        } else if (ip == 4) {
            dOk = 1;
        }
        double dI[3];
        for (int iw = 0; iw < 3; iw++) {
            dI[iw] = 0;
            for (int ig = 0; ig < 5; ig++) dI[iw] += cg[ig] * Iv[3 + 5 * iw + ig];
        }
        double ddM = DH * (SD * dI[0] + Sk * dOk);
        J[0 * ncol + ip] = DH * dI[0];
        J[1 * ncol + ip] = tH * dI[1];
        J[2 * ncol + ip] = DH * dI[2];
        J[3 * ncol + ip] = ddM;
        J[4 * ncol + ip] = lf * ddM;
        J[5 * ncol + ip] = (z2 == z1) ? 0.0 : 5.0 / log(10.0) * ddM / dM;
    }
}

/* O1 (+ O4 when jac != NULL), z1 = 0 and z2 = z for every pair.
 * params [B][ncol] = (H0, Om, OL, Or[, Ok]); z [nnz]; rows by offsets.
 * out [nnz][6] = (d_C, t, X, d_M, d_L, mu) in Mpc / Gyr / mag.
 * jac [nnz][6][ncol]: d out / d params (H0 first).
 * Returns 0 on success. */
int oracle_quad_distances(const double* params, int64_t B, int ncol, const int64_t* offsets,
                          const double* z, int64_t nnz, double rtol, double* out, double* jac) {
    if (!gl_ready) gl_init();
    for (int64_t j = 0; j < nnz; j++) {
        int64_t b = row_of(offsets, B, nnz, j);
        double H0;
        cosmo_t c;
        unpack_params(params + b * ncol, ncol, &H0, &c);
        quad_pair(&c, H0, ncol, 0.0, z[j], rtol, out + 6 * j, jac ? jac + 6 * ncol * j : NULL);
    }
    return 0;
}

/* O1 (+ O4) with general limits (eqs. 2.3-2.5 as defined, z1 <= z2): the
 * lower limit z1[b] per row, the upper limit z2[j] per pair; outputs as in
 * quad_pair.  Pairs with z2 < z1 give NaN. */
int oracle_quad_between(const double* params, int64_t B, int ncol, const int64_t* offsets, const double* z1,
                        const double* z2, int64_t nnz, double rtol, double* out, double* jac) {
    if (!gl_ready) gl_init();
    for (int64_t j = 0; j < nnz; j++) {
        int64_t b = row_of(offsets, B, nnz, j);
        double H0;
        cosmo_t c;
        unpack_params(params + b * ncol, ncol, &H0, &c);
        if (!(z2[j] >= z1[b])) {
            for (int k = 0; k < 6; k++) out[6 * j + k] = NAN;
            if (jac) for (int k = 0; k < 6 * ncol; k++) jac[6 * ncol * j + k] = NAN;
            continue;
        }
        quad_pair(&c, H0, ncol, z1[b], z2[j], rtol, out + 6 * j, jac ? jac + 6 * ncol * j : NULL);
    }
    return 0;
}

/* O1 (+ O4) for the upper limit z2 -> infinity, per row b with lower limit
 * z1[b] (Sec. 2.1.1: the age of the universe at z1 is t(z1, infinity)):
 * out [B][2] = (chi(z1, inf) [Mpc], the comoving distance to the particle
 * horizon; t(z1, inf) [Gyr], the age), jac [B][2][ncol]. */
int oracle_quad_limits(const double* params, int64_t B, int ncol, const double* z1, double rtol, double* out,
                       double* jac) {
    if (!gl_ready) gl_init();
    for (int64_t b = 0; b < B; b++) {
        double H0;
        cosmo_t c;
        unpack_params(params + b * ncol, ncol, &H0, &c);
        double DH = C_KMS / H0, tH = HUBBLE_TIME_GYR / H0, Iv[NCOMP];
        integrate_between(&c, z1[b], INFINITY, rtol, KMASK_NO_X & kmask_for(ncol), Iv);
        out[2 * b] = DH * Iv[0];
        out[2 * b + 1] = tH * Iv[1];
        if (!jac) continue;
        double* J = jac + 2 * ncol * b;
        J[0] = -out[2 * b] / H0;
        J[ncol] = -out[2 * b + 1] / H0;
        for (int ip = 1; ip < ncol; ip++) {
            double cg[5] = {0, 0, 0, 0, 0};
            cg[ip <= 4 ? ip - 1 : (ip == 5 ? 3 : 4)] = 1;
            if (ncol == 4) cg[3] = -1;
            double d0 = 0, d1 = 0;
            for (int ig = 0; ig < 5; ig++) { d0 += cg[ig] * Iv[3 + ig]; d1 += cg[ig] * Iv[8 + ig]; }
            J[ip] = DH * d0;
            J[ncol + ip] = tH * d1;
        }
    }
    return 0;
}

/* ======================================================================== */
/* O2: Carlson formulas (3.7)-(3.9) and (B.1)-(B.3) for limits z1 <= z2,    */
/* with X_m = sqrt(z2 - r_m), Y_m = sqrt(z1 - r_m) and Delta z = z2 - z1     */
/* as defined in Sec. 3.1; and their limits as z2 -> infinity.              */
/* ======================================================================== */

/* Y_m = sqrt(z1 - r_m) (mutation 7 drops z1 here) */
static cplx lower_root(double z1, cplx r) { return csqrt((g_mutation == 7 ? 0.0 : z1) - r); }

/* Quartic, eqs. (3.7)-(3.9).  r[4]: roots of E^2 in z.  it: index i for t;
 * (iX, lX): indices i and l for X; the remaining two are j, k.  Outputs
 * chi, t, X in units of c/H0, 1/H0, c/H0 with the Or^-1/2 prefactor
 * included; im[3] receives the imaginary parts (should vanish). */
static void quartic_carlson(const cplx* r, double Or, double z1, double z2, int it, int iX, int lX,
                            double* res, double* im) {
    cplx X[4], Y[4];
    const double dz = z2 - z1;
    for (int m = 0; m < 4; m++) {
        X[m] = csqrt(z2 - r[m]);
        Y[m] = lower_root(z1, r[m]);
        if (g_mutation == 3) { cplx s = X[m]; X[m] = Y[m]; Y[m] = s; }
    }
    /* u_ab = X_a X_b Y_c Y_d + Y_a Y_b X_c X_d, {c,d} the complement of {a,b} */
#define UAB(a, b, out) do { int cc_ = -1, dd_ = -1; \
        for (int m_ = 0; m_ < 4; m_++) if (m_ != (a) && m_ != (b)) { if (cc_ < 0) cc_ = m_; else dd_ = m_; } \
        out = X[a] * X[b] * Y[cc_] * Y[dd_] + Y[a] * Y[b] * X[cc_] * X[dd_]; } while (0)
    cplx Ut[3];
    double Or_h = 1.0 / sqrt(Or);
    /* ---- chi, eq. (3.7): R_F of (u_12^2, u_13^2, u_14^2) ---- */
    cplx u12, u13, u14;
    UAB(0, 1, u12); UAB(0, 2, u13); UAB(0, 3, u14);
    cplx rf = oracle_rf(u12 * u12, u13 * u13, u14 * u14);
    cplx chi = Or_h * 2.0 * dz * rf;
    /* ---- t, eq. (3.8), with the index i = it ---- */
    {
        int i = it, o[3], n = 0;
        for (int m = 0; m < 4; m++) if (m != i) o[n++] = m;
        int j = o[0], k = o[1], l = o[2];
        cplx uij, uik, uil;
        UAB(i, j, uij); UAB(i, k, uik); UAB(i, l, uil);
        Ut[0] = uij * uij; Ut[1] = uik * uik; Ut[2] = uil * uil;
        cplx dij = r[j] - r[i], dik = r[k] - r[i], dil = r[l] - r[i];
        cplx di5 = -(1.0 + r[i]), dj5 = -(1.0 + r[j]), dk5 = -(1.0 + r[k]), dl5 = -(1.0 + r[l]);
        cplx ui5 = Ut[0] - dz * dz * dik * dil * dj5 / di5;
        cplx qi5 = (z1 + 1.0) * (z2 + 1.0) / ((z1 - r[i]) * (z2 - r[i])) * ui5;
        cplx si5 = qi5 + dz * dz * dk5 * dl5 * dj5 / di5;
        if (fabs(cimag(ui5)) <= 1e-13 * cabs(ui5)) ui5 = creal(ui5);
        if (fabs(cimag(qi5)) <= 1e-13 * cabs(qi5)) qi5 = creal(qi5);
        if (fabs(cimag(si5)) <= 1e-13 * cabs(si5)) si5 = creal(si5);
        cplx rfi = oracle_rf(Ut[0], Ut[1], Ut[2]);
        cplx br = dz * dz / 3.0 * dij * dik * dil / di5 * oracle_rj(Ut[0], Ut[1], Ut[2], ui5)
                  + (g_mutation == 2 ? -1.0 : 1.0) * oracle_rc(si5, qi5);
        cplx t = Or_h * 2.0 * dz / (r[i] + 1.0) * (rfi - br);
        res[1] = creal(t); im[1] = cimag(t);
    }
    /* ---- X, eq. (3.9), with indices i = iX, l = lX ---- */
    {
        int i = iX, l = lX, o[2], n = 0;
        for (int m = 0; m < 4; m++) if (m != i && m != l) o[n++] = m;
        int j = o[0], k = o[1];
        cplx uij, uik, uil;
        UAB(i, j, uij); UAB(i, k, uik); UAB(i, l, uil);
        cplx U0 = uij * uij, U1 = uik * uik, U2 = uil * uil;
        cplx dij = r[j] - r[i], dik = r[k] - r[i], dil = r[l] - r[i];
        cplx djl = r[l] - r[j], dkl = r[l] - r[k];
        cplx ui0 = U0 - dz * dz * dik * dil;
        cplx qi0 = ui0 / ((z1 - r[i]) * (z2 - r[i]));
        cplx si0 = qi0 + dz * dz;
        if (fabs(cimag(ui0)) <= 1e-13 * cabs(ui0)) ui0 = creal(ui0);
        if (fabs(cimag(qi0)) <= 1e-13 * cabs(qi0)) qi0 = creal(qi0);
        if (fabs(cimag(si0)) <= 1e-13 * cabs(si0)) si0 = creal(si0);
        cplx sumr = r[0] + r[1] + r[2] + r[3] + 4.0;
        cplx rfx = oracle_rf(U0, U1, U2);
        cplx term0 = (X[i] * X[j] * X[k] / X[l] - Y[i] * Y[j] * Y[k] / Y[l]) / dz;
        cplx term1 = (2.0 * (r[i] + 1.0) * (r[i] + 1.0) - dij * dik) * rfx;
        cplx term2 = djl * dkl * (dz * dz / 3.0 * dij * dik * oracle_rd(U0, U1, U2)
                                  + X[i] * Y[i] / (X[l] * Y[l]) / uil);
        cplx term3 = sumr * (dz * dz / 3.0 * dij * dik * dil / (-1.0) * oracle_rj(U0, U1, U2, ui0)
                             + oracle_rc(si0, qi0));
        cplx Xd = Or_h * dz * (term0 + term1 + term2 + term3);
        res[2] = creal(Xd); im[2] = cimag(Xd);
    }
    res[0] = creal(chi); im[0] = cimag(chi);
#undef UAB
}

/* Cubic (Or = 0), eqs. (B.1)-(B.3); r[3] roots of E^2 in z, i = index i. */
static void cubic_carlson(const cplx* r, double Om, double z1, double z2, int i, double* res, double* im) {
    cplx X[3], Y[3];
    const double dz = z2 - z1;
    for (int m = 0; m < 3; m++) {
        X[m] = csqrt(z2 - r[m]);
        Y[m] = lower_root(z1, r[m]);
        if (g_mutation == 3) { cplx s = X[m]; X[m] = Y[m]; Y[m] = s; }
    }
    cplx u[3];
    for (int a = 0; a < 3; a++) {
        int b = (a + 1) % 3, c = (a + 2) % 3;
        u[a] = X[a] * Y[b] * Y[c] + Y[a] * X[b] * X[c];
    }
    int j = (i + 1) % 3, k = (i + 2) % 3;
    cplx U[3] = {u[0] * u[0], u[1] * u[1], u[2] * u[2]};
    double Om_h = 1.0 / sqrt(Om);
    cplx rf = oracle_rf(U[0], U[1], U[2]);
    cplx chi = Om_h * 2.0 * dz * rf;
    cplx ui5 = U[i] + dz * dz * (r[i] + 1.0);
    cplx s5 = Y[0] * Y[1] * Y[2] * (z2 + 1.0) + X[0] * X[1] * X[2] * (z1 + 1.0);
    cplx qi5 = (z1 + 1.0) * (z2 + 1.0) * ui5;
    if (fabs(cimag(ui5)) <= 1e-13 * cabs(ui5)) ui5 = creal(ui5);
    if (fabs(cimag(qi5)) <= 1e-13 * cabs(qi5)) qi5 = creal(qi5);
    cplx s52 = s5 * s5;
    if (fabs(cimag(s52)) <= 1e-13 * cabs(s52)) s52 = creal(s52);
    cplx t = Om_h * 2.0 * dz * (dz * dz / 3.0 * oracle_rj(U[0], U[1], U[2], ui5)
                                + (g_mutation == 2 ? -1.0 : 1.0) * oracle_rc(s52, qi5));
    cplx dij = r[j] - r[i], dik = r[k] - r[i];
    cplx sumr = r[0] + r[1] + r[2] + 3.0;
    cplx Xd = Om_h * 2.0 * dz / 3.0 *
              ((X[0] * X[1] * X[2] - Y[0] * Y[1] * Y[2]) / dz
               + (3.0 * (r[i] + 1.0) * (r[i] + 1.0) - dij * dik) * rf
               + 2.0 * sumr * (dz * dz / 3.0 * dij * dik * oracle_rd(U[j], U[k], U[i])
                               + Y[i] * X[i] / u[i]));
    res[0] = creal(chi); im[0] = cimag(chi);
    res[1] = creal(t); im[1] = cimag(t);
    res[2] = creal(Xd); im[2] = cimag(Xd);
}

/* The z2 -> infinity limits of eqs. (3.7) and (3.8) (quartic, index i = it
 * for t).  With X_m ~ sqrt(z2) every u_ab grows like Delta z, and
 *   U_ab = lim u_ab / Delta z = Y_c Y_d + Y_a Y_b
 * ({c,d} the complement of {a,b}); R_F and R_C are homogeneous of degree
 * -1/2 and R_J of degree -3/2, so every Delta z prefactor cancels:
 *   chi(z1, inf) = Or^-1/2 2 R_F(U_12^2, U_13^2, U_14^2),
 *   t(z1, inf)   = Or^-1/2 2/(r_i+1) { R_F - [ d_ij d_ik d_il/(3 d_i5)
 *                  R_J(..., U_i5^2) + R_C(S_i5^2, Q_i5^2) ] },
 *   U_i5^2 = U_ij^2 - d_ik d_il d_j5/d_i5,  Q_i5^2 = (z1+1)/(z1-r_i) U_i5^2,
 *   S_i5^2 = Q_i5^2 + d_k5 d_l5 d_j5/d_i5.
 * res[2] = (chi, t) in units of c/H0 and 1/H0. */
static void quartic_carlson_inf(const cplx* r, double Or, double z1, int it, double* res, double* im) {
    cplx Y[4];
    for (int m = 0; m < 4; m++) Y[m] = lower_root(z1, r[m]);
#define UINF(a, b, out) do { int cc_ = -1, dd_ = -1; \
        for (int m_ = 0; m_ < 4; m_++) if (m_ != (a) && m_ != (b)) { if (cc_ < 0) cc_ = m_; else dd_ = m_; } \
        out = Y[cc_] * Y[dd_] + Y[a] * Y[b]; } while (0)
    double Or_h = 1.0 / sqrt(Or);
    cplx u12, u13, u14;
    UINF(0, 1, u12); UINF(0, 2, u13); UINF(0, 3, u14);
    cplx chi = Or_h * 2.0 * oracle_rf(u12 * u12, u13 * u13, u14 * u14);
    int i = it, o[3], n = 0;
    for (int m = 0; m < 4; m++) if (m != i) o[n++] = m;
    int j = o[0], k = o[1], l = o[2];
    cplx uij, uik, uil;
    UINF(i, j, uij); UINF(i, k, uik); UINF(i, l, uil);
    cplx U0 = uij * uij, U1 = uik * uik, U2 = uil * uil;
    cplx dij = r[j] - r[i], dik = r[k] - r[i], dil = r[l] - r[i];
    cplx di5 = -(1.0 + r[i]), dj5 = -(1.0 + r[j]), dk5 = -(1.0 + r[k]), dl5 = -(1.0 + r[l]);
    cplx ui5 = U0 - dik * dil * dj5 / di5;
    cplx qi5 = (z1 + 1.0) / (z1 - r[i]) * ui5;
    cplx si5 = qi5 + dk5 * dl5 * dj5 / di5;
    if (fabs(cimag(ui5)) <= 1e-13 * cabs(ui5)) ui5 = creal(ui5);
    if (fabs(cimag(qi5)) <= 1e-13 * cabs(qi5)) qi5 = creal(qi5);
    if (fabs(cimag(si5)) <= 1e-13 * cabs(si5)) si5 = creal(si5);
    cplx br = dij * dik * dil / (3.0 * di5) * oracle_rj(U0, U1, U2, ui5)
              + (g_mutation == 8 ? 0.0 : 1.0) * oracle_rc(si5, qi5);
    cplx t = Or_h * 2.0 / (r[i] + 1.0) * (oracle_rf(U0, U1, U2) - br);
    res[0] = creal(chi); im[0] = cimag(chi);
    res[1] = creal(t); im[1] = cimag(t);
#undef UINF
}

/* The z2 -> infinity limits of eqs. (B.1) and (B.2).  Here u_i / Delta z ->
 * Y_i, so U_i^2 = z1 - r_i and U_i5^2 = U_i^2 + (r_i + 1) = 1 + z1; the R_C
 * term of (B.2) falls off like Delta z^-1/2 and vanishes:
 *   chi(z1, inf) = Om^-1/2 2 R_F(z1 - r_1, z1 - r_2, z1 - r_3),
 *   t(z1, inf)   = Om^-1/2 (2/3) R_J(z1 - r_1, z1 - r_2, z1 - r_3, 1 + z1). */
static void cubic_carlson_inf(const cplx* r, double Om, double z1, int i, double* res, double* im) {
    cplx Y[3], U[3];
    for (int m = 0; m < 3; m++) { Y[m] = lower_root(z1, r[m]); U[m] = Y[m] * Y[m]; }
    double Om_h = 1.0 / sqrt(Om);
    cplx chi = Om_h * 2.0 * oracle_rf(U[0], U[1], U[2]);
    cplx ui5 = U[i] + (r[i] + 1.0);
    if (fabs(cimag(ui5)) <= 1e-13 * cabs(ui5)) ui5 = creal(ui5);
    cplx t = Om_h * 2.0 / 3.0 * oracle_rj(U[0], U[1], U[2], ui5);
    res[0] = creal(chi); im[0] = cimag(chi);
    res[1] = creal(t); im[1] = cimag(t);
}

static void unpack_roots(const double* roots, int64_t b, int m, cplx* r) {
    for (int a = 0; a < m; a++) r[a] = (roots[8 * b + 2 * a] - 1.0) + I * roots[8 * b + 2 * a + 1];
}

/* O2 batch with general limits.  roots [B][4] complex (re,im) of E^2 in
 * x = 1+z (Sec. 3, eq. 3.2; m = nroot[b] = 4 or 3 entries used); perm [B][3]
 * = (i_t, i_X, l_X); z1 [B] lower limits (NULL: 0), z2 [nnz] upper limits.
 * out [nnz][6] as in quad_pair; imag [nnz][3] imaginary parts. */
int oracle_carlson_between(const double* params, int64_t B, int ncol, const int64_t* offsets,
                           const double* z1v, const double* z, int64_t nnz, const double* roots,
                           const int32_t* nroot, const int32_t* perm, double* out, double* imag) {
    for (int64_t j = 0; j < nnz; j++) {
        int64_t b = row_of(offsets, B, nnz, j);
        double H0;
        cosmo_t c;
        unpack_params(params + b * ncol, ncol, &H0, &c);
        double z1 = z1v ? z1v[b] : 0.0, zz = z[j], DH = C_KMS / H0, tH = HUBBLE_TIME_GYR / H0;
        double* o = out + 6 * j;
        if (!(zz >= z1)) {
            for (int k = 0; k < 6; k++) o[k] = NAN;
            if (imag) for (int k = 0; k < 3; k++) imag[3 * j + k] = NAN;
            continue;
        }
        int m = nroot[b];
        cplx r[4];
        unpack_roots(roots, b, m, r);
        double res[3] = {0, 0, 0}, im[3] = {0, 0, 0};
        if (zz != z1) {
            if (m == 4)
                quartic_carlson(r, c.Or, z1, zz, perm[3 * b], perm[3 * b + 1], perm[3 * b + 2], res, im);
            else
                cubic_carlson(r, c.Om, z1, zz, perm[3 * b + 1], res, im);
        }
        double S, SD, Sk;
        curv_map(res[0], c.Ok, &S, &SD, &Sk);
        o[0] = DH * res[0]; o[1] = tH * res[1]; o[2] = DH * res[2];
        o[3] = DH * S;
        o[4] = (g_mutation == 4 ? 1.0 : 1.0 + zz) / ((1.0 + z1) * (1.0 + z1)) * o[3];
        o[5] = 5.0 * log10(o[4]) + 25.0;
        if (imag) { imag[3 * j] = DH * im[0]; imag[3 * j + 1] = tH * im[1]; imag[3 * j + 2] = DH * im[2]; }
    }
    return 0;
}

/* O2 with z1 = 0, z2 = z for every pair. */
int oracle_carlson_distances(const double* params, int64_t B, int ncol, const int64_t* offsets,
                             const double* z, int64_t nnz, const double* roots,
                             const int32_t* nroot, const int32_t* perm, double* out,
                             double* imag) {
    return oracle_carlson_between(params, B, ncol, offsets, NULL, z, nnz, roots, nroot, perm, out, imag);
}

/* O2 limits z2 -> infinity per row: out [B][2] = (chi(z1, inf) [Mpc],
 * t(z1, inf) [Gyr]); imag [B][2] imaginary parts (may be NULL). */
int oracle_carlson_limits(const double* params, int64_t B, int ncol, const double* z1v, const double* roots,
                          const int32_t* nroot, const int32_t* perm, double* out, double* imag) {
    for (int64_t b = 0; b < B; b++) {
        double H0;
        cosmo_t c;
        unpack_params(params + b * ncol, ncol, &H0, &c);
        int m = nroot[b];
        cplx r[4];
        unpack_roots(roots, b, m, r);
        double res[2], im[2];
        if (m == 4)
            quartic_carlson_inf(r, c.Or, z1v[b], perm[3 * b], res, im);
        else
            cubic_carlson_inf(r, c.Om, z1v[b], perm[3 * b + 1], res, im);
        out[2 * b] = C_KMS / H0 * res[0];
        out[2 * b + 1] = HUBBLE_TIME_GYR / H0 * res[1];
        if (imag) { imag[2 * b] = C_KMS / H0 * im[0]; imag[2 * b + 1] = HUBBLE_TIME_GYR / H0 * im[1]; }
    }
    return 0;
}

/* Fine-grid composite Simpson rule of the same three integrals (brute force
 * check for tiny inputs): n even subintervals on [1/(1+z), 1]. */
int oracle_simpson(const double* p, int ncol, double z, int64_t n, double* res) {
    double H0;
    cosmo_t c;
    unpack_params(p, ncol, &H0, &c);
    double lo = 1.0 / (1.0 + z), h = (1.0 - lo) / n, s[3] = {0, 0, 0}, v[NCOMP];
    for (int64_t i = 0; i <= n; i++) {
        double w = (i == 0 || i == n) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
        integrand(lo + i * h, &c, v);
        for (int k = 0; k < 3; k++) s[k] += w * v[k];
    }
    res[0] = C_KMS / H0 * s[0] * h / 3.0;
    res[1] = HUBBLE_TIME_GYR / H0 * s[1] * h / 3.0;
    res[2] = C_KMS / H0 * s[2] * h / 3.0;
    return 0;
}

/* ======================================================================== */
/* Comparators of the speed study (Sec. 3.2.2, Fig. 3): the Legendre form  */
/* of App. B.2 and the hypergeometric solution of the flat radiationless   */
/* comoving distance.  FP64, plain; used for timing beside O1 and O2 and   */
/* pinned against O1.                                                      */
/* ======================================================================== */

/* Legendre's integrals with c = csc^2 phi (App. B.2's tilde notation), from
 * Carlson's (DLMF 19.25.5 and 19.25.14):
 *   F~(c, m)    = R_F(c - 1, c - m, c),
 *   Pi~(n, c, m) = F~(c, m) + (n/3) R_J(c - 1, c - m, c, c - n). */
static cplx leg_F(cplx c, cplx m) { return oracle_rf(c - 1.0, c - m, c); }
static cplx leg_Pi(cplx n, cplx c, cplx m) {
    return leg_F(c, m) + n / 3.0 * oracle_rj(c - 1.0, c - m, c, c - n);
}

/* eqs. (B.4)-(B.5) (quartic, roots r[0..3] in z, assignment i j k l) and
 * (B.6)-(B.7) (cubic, r[0..2], assignment i j k) for one pair, z1 -> z2;
 * res = (chi H0/c, t H0) without the alpha_m^-1/2 prefactor, complex.  The
 * bracket [f]_{z2}^{z1} is f(z1) - f(z2), as printed. */
static void legendre_pair(const cplx* r, int nroot, const int* ijkl, double z1, double z2, cplx* chi, cplx* t) {
    const int i = ijkl[0], j = ijkl[1], k = ijkl[2], l = ijkl[3];
    if (nroot == 4) {
        cplx m = (r[k] - r[j]) / (r[k] - r[i]) * (r[l] - r[i]) / (r[l] - r[j]);
        cplx n = (1.0 + r[j]) / (1.0 + r[i]) * (r[l] - r[i]) / (r[l] - r[j]);
        cplx c1 = (z1 - r[j]) / (z1 - r[i]) * (r[l] - r[i]) / (r[l] - r[j]);
        cplx c2 = (z2 - r[j]) / (z2 - r[i]) * (r[l] - r[i]) / (r[l] - r[j]);
        cplx den = csqrt((r[i] - r[k]) * (r[j] - r[l]));
        *chi = 2.0 * (leg_F(c1, m) - leg_F(c2, m)) / den;
        cplx b1 = (1.0 + r[i]) * leg_F(c1, m) - (r[i] - r[j]) * leg_Pi(n, c1, m);
        cplx b2 = (1.0 + r[i]) * leg_F(c2, m) - (r[i] - r[j]) * leg_Pi(n, c2, m);
        *t = 2.0 * (b1 - b2) / (den * (1.0 + r[i]) * (1.0 + r[j]));
    } else {
        cplx m = (r[k] - r[i]) / (r[j] - r[i]);
        cplx n = -(1.0 + r[i]) / (r[j] - r[i]);
        cplx c1 = (z1 - r[i]) / (r[j] - r[i]), c2 = (z2 - r[i]) / (r[j] - r[i]);
        cplx den = csqrt(r[j] - r[i]);
        *chi = 2.0 * (leg_F(c1, m) - leg_F(c2, m)) / den;
        /* (B.7) with its prefactor read as 1/H0 (a time) */
        *t = 2.0 * ((leg_F(c1, m) - leg_Pi(n, c1, m)) - (leg_F(c2, m) - leg_Pi(n, c2, m))) / (den * (1.0 + r[i]));
    }
}

/* Batch: pairs of rows b with roots[b][4] (complex, in x = 1 + z as for O2),
 * nroot[b] and assignment ijkl[b][4]; out[p][2] = (d_C [Mpc], t [Gyr]). */
int oracle_legendre_distances(const double* params, int64_t B, int ncol, const int64_t* offsets, const double* z,
                              int64_t nnz, const double* roots, const int32_t* nroot, const int32_t* ijkl,
                              double* out) {
    (void)nnz;
    for (int64_t b = 0; b < B; b++) {
        const double H0 = params[b * ncol], Om = params[b * ncol + 1], Or = params[b * ncol + 3];
        cplx r[4];
        for (int m = 0; m < 4; m++) r[m] = roots[(b * 4 + m) * 2] - 1.0 + I * roots[(b * 4 + m) * 2 + 1];
        const int q[4] = {ijkl[4 * b], ijkl[4 * b + 1], ijkl[4 * b + 2], ijkl[4 * b + 3]};
        const double pre = 1.0 / sqrt(nroot[b] == 4 ? Or : Om);
        for (int64_t p = offsets[b]; p < offsets[b + 1]; p++) {
            cplx chi, t;
            legendre_pair(r, nroot[b], q, 0.0, z[p], &chi, &t);
            out[2 * p] = creal(chi) * pre * C_KMS / H0;
            out[2 * p + 1] = creal(t) * pre * HUBBLE_TIME_GYR / H0;
        }
    }
    return 0;
}

/* Gauss's hypergeometric series 2F1(a, b; c; u) for 0 <= u <= 1/2. */
static double hyp2f1_series(double a, double b, double c, double u) {
    double term = 1.0, sum = 1.0;
    for (int n = 0; n < 2000; n++) {
        term *= (a + n) * (b + n) / ((c + n) * (n + 1.0)) * u;
        sum += term;
        if (fabs(term) <= 1e-17 * fabs(sum)) break;
    }
    return sum;
}

/* The flat radiationless comoving distance by the hypergeometric function
 * (Sec. 3.2.2 and its ref. [2]):
 *   int dx / sqrt(OL + Om x^3) = x 2F1(1/2, 1/3; 4/3; -(Om/OL) x^3) / sqrt(OL),
 * with 2F1(1/2, 1/3; 4/3; -y) = (1+y)^(-1/3) 2F1(5/6, 1/3; 4/3; u),
 * u = y/(1+y) (Pfaff, DLMF 15.8.1), summed directly for u <= 1/2 and through
 * the connection to 1 - u (DLMF 15.8.4; c - a - b = 1/6) otherwise:
 *   2F1(5/6, 1/3; 4/3; u) = G1 u^(-1/3) + G2 (1-u)^(1/6) 2F1(1/2, 1; 7/6; 1 - u),
 *   G1 = G(4/3) G(1/6) / (G(1/2) G(1)),  G2 = G(4/3) G(-1/6) / (G(5/6) G(1/3)). */
static double f21_flat(double y) {
    const double u = y / (1.0 + y), v = 1.0 / (1.0 + y);   /* v = 1 - u, formed without cancellation */
    double f;
    if (u <= 0.5) {
        f = hyp2f1_series(5.0 / 6.0, 1.0 / 3.0, 4.0 / 3.0, u);
    } else {
        const double G1 = tgamma(4.0 / 3.0) * tgamma(1.0 / 6.0) / (tgamma(0.5) * tgamma(1.0));
        const double G2 = tgamma(4.0 / 3.0) * tgamma(-1.0 / 6.0) / (tgamma(5.0 / 6.0) * tgamma(1.0 / 3.0));
        f = G1 * pow(u, -1.0 / 3.0) + G2 * pow(v, 1.0 / 6.0) * hyp2f1_series(0.5, 1.0, 7.0 / 6.0, v);
    }
    return pow(1.0 + y, -1.0 / 3.0) * f;
}

/* d_C [Mpc] of the flat radiationless cosmology (H0, Om, OL = 1 - Om) at z[n]. */
int oracle_hyp2f1_flat(double H0, double Om, const double* z, int64_t n, double* out) {
    const double OL = 1.0 - Om, w = Om / OL;
    const double f1 = f21_flat(w);
    for (int64_t p = 0; p < n; p++) {
        const double x = 1.0 + z[p];
        out[p] = (x * f21_flat(w * x * x * x) - f1) / sqrt(OL) * C_KMS / H0;
    }
    return 0;
}
