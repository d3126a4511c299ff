// Device arithmetic for the Carlson-integral distance path.
//
//  * df64        double-float numbers (an unevaluated sum of two floats,
//                Dekker/Knuth error-free transformations), used for the
//                per-lane accumulators of the reductions (GB300 issues about
//                1.6 DFMA per SM per clock against about 115 FFMA).
//  * Dual<T,K>   value + K tangents (forward mode over the density parameters).
//  * Cx<S>       complex numbers over any scalar S.
//  * CPair/RPair the two roots (or integral arguments) that are either a complex
//                conjugate pair or two reals, with the operations the formulas
//                need (sum and product of the members are real in both cases).
//  * carlson_sym one duplication sequence on (x1, y_a, y_b) shared by R_F,
//                R_D (x1 special) and up to two R_J tracks (eqs. 2.6-2.9),
//                after Carlson's duplication algorithm (the paper's ref. [10]),
//                carried on the pair's symmetric functions, and optionally the
//                divided difference of the last R_J track against R_D; generic
//                over plain and dual numbers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

// Function qualifiers (overridable: the arithmetic is plain C++ and also
// compiles for the host).
#ifndef LCDM_HD
#define LCDM_HD __device__ __forceinline__
#endif
// Routines off the main path (R_C by duplication and its fallbacks) are real
// calls, compiled once per instantiation.  The main path (the integrals and
// the shared duplication sequence) is inlined into the kernels: with the
// kernels' register caps the allocator then sees the whole pair at once,
// with no argument passing through local memory (measured faster).
#ifndef LCDM_NI
#define LCDM_NI __device__ __noinline__
#endif
// round-to-nearest float add / sub that the compiler may not contract
#ifdef __CUDA_ARCH__
#define LCDM_FADD(a, b) __fadd_rn(a, b)
#define LCDM_FSUB(a, b) __fsub_rn(a, b)
#else
#define LCDM_FADD(a, b) ((a) + (b))
#define LCDM_FSUB(a, b) ((a) - (b))
#endif

namespace lcdm {

// ---------------------------------------------------------------------------
// df64: a float pair (hi + lo) used as the per-lane accumulator of the
// per-cosmology sums in the FP32 path (no FP64 arithmetic per pair).
// ---------------------------------------------------------------------------
struct df64 {
    float hi, lo;
};
LCDM_HD df64 mkdf(float h, float l = 0.f) { df64 r; r.hi = h; r.lo = l; return r; }
LCDM_HD df64 df_from_double(double d) { float h = (float)d; return mkdf(h, (float)(d - (double)h)); }
// error-free sum (Knuth), sum with |a| >= |b| (Dekker)
LCDM_HD df64 two_sum(float a, float b) {
    float s = LCDM_FADD(a, b), bb = LCDM_FSUB(s, a);
    float e = LCDM_FADD(LCDM_FSUB(a, LCDM_FSUB(s, bb)), LCDM_FSUB(b, bb));
    return mkdf(s, e);
}
LCDM_HD df64 fast_two_sum(float a, float b) {
    float s = LCDM_FADD(a, b);
    return mkdf(s, LCDM_FSUB(b, LCDM_FSUB(s, a)));
}
LCDM_HD df64 operator+(df64 a, df64 b) {
    df64 s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
    s.lo = LCDM_FADD(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = LCDM_FADD(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}
// a + b for a plain float b: one error-free sum of the high words, the low
// word and the rounding error added, renormalised (about half the work of the
// double-float sum)
LCDM_HD df64 operator+(df64 a, float b) {
    df64 s = two_sum(a.hi, b);
    s.lo = LCDM_FADD(s.lo, a.lo);
    return fast_two_sum(s.hi, s.lo);
}

// ---------------------------------------------------------------------------
// Scalar traits: value used for branching, sqrt, abs, constants.
// ---------------------------------------------------------------------------
LCDM_HD float sval(float a) { return a; }
LCDM_HD double sval(double a) { return a; }
LCDM_HD float ssqrt(float a) { return sqrtf(a); }
LCDM_HD double ssqrt(double a) { return sqrt(a); }
LCDM_HD float sabs(float a) { return fabsf(a); }
LCDM_HD double sabs(double a) { return fabs(a); }
template <class T> struct CstImpl;
template <> struct CstImpl<float> { static LCDM_HD float make(double v) { return (float)v; } };
template <> struct CstImpl<double> { static LCDM_HD double make(double v) { return v; } };
template <> struct CstImpl<df64> { static LCDM_HD df64 make(double v) { return df_from_double(v); } };
template <class T> LCDM_HD T cst(double v) { return CstImpl<T>::make(v); }
// exact multiplication by 2^e

// ---------------------------------------------------------------------------
// Dual numbers (forward-mode tangents over K parameters)
// ---------------------------------------------------------------------------
template <class T, int K>
struct Dual {
    T v;
    T d[K];
};
template <class T, int K> LCDM_HD Dual<T, K> dconst(T v) {
    Dual<T, K> r; r.v = v;
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = cst<T>(0.0);
    return r;
}
template <class T, int K> LCDM_HD Dual<T, K> operator+(const Dual<T, K>& a, const Dual<T, K>& b) {
    Dual<T, K> r; r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = a.d[k] + b.d[k];
    return r;
}
template <class T, int K> LCDM_HD Dual<T, K> operator-(const Dual<T, K>& a, const Dual<T, K>& b) {
    Dual<T, K> r; r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = a.d[k] - b.d[k];
    return r;
}
template <class T, int K> LCDM_HD Dual<T, K> operator-(const Dual<T, K>& a) {
    Dual<T, K> r; r.v = -a.v;
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = -a.d[k];
    return r;
}
template <class T, int K> LCDM_HD Dual<T, K> operator*(const Dual<T, K>& a, const Dual<T, K>& b) {
    Dual<T, K> r; r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
template <class T, int K> LCDM_HD Dual<T, K> operator/(const Dual<T, K>& a, const Dual<T, K>& b) {
    Dual<T, K> r; T ib = cst<T>(1.0) / b.v; r.v = a.v * ib;
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
}
template <class T, int K> LCDM_HD Dual<T, K> operator+(const Dual<T, K>& a, T b) { Dual<T, K> r = a; r.v = a.v + b; return r; }
template <class T, int K> LCDM_HD Dual<T, K> operator+(T b, const Dual<T, K>& a) { return a + b; }
template <class T, int K> LCDM_HD Dual<T, K> operator-(const Dual<T, K>& a, T b) { Dual<T, K> r = a; r.v = a.v - b; return r; }
template <class T, int K> LCDM_HD Dual<T, K> operator-(T b, const Dual<T, K>& a) { return (-a) + b; }
template <class T, int K> LCDM_HD Dual<T, K> operator*(const Dual<T, K>& a, T b) {
    Dual<T, K> r; r.v = a.v * b;
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = a.d[k] * b;
    return r;
}
template <class T, int K> LCDM_HD Dual<T, K> operator*(T b, const Dual<T, K>& a) { return a * b; }
template <class T, int K> LCDM_HD Dual<T, K> operator/(const Dual<T, K>& a, T b) { return a * (cst<T>(1.0) / b); }
template <class T, int K> LCDM_HD Dual<T, K> operator/(T a, const Dual<T, K>& b) { return dconst<T, K>(a) / b; }
template <class T, int K> LCDM_HD T sval(const Dual<T, K>& a) { return a.v; }
template <class T, int K> LCDM_HD Dual<T, K> ssqrt(const Dual<T, K>& a) {
    Dual<T, K> r; r.v = ssqrt(a.v);
    T h = cst<T>(0.5) / r.v;
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = a.d[k] * h;
    return r;
}
// FP32: one reciprocal square root gives both the value (a rsqrt(a)) and the
// tangents' factor (rsqrt(a)/2), one special-function operation instead of two
LCDM_HD float srsqrt(float a) {
#ifdef __CUDA_ARCH__
    return rsqrtf(a);
#else
    return 1.0f / sqrtf(a);
#endif
}
template <int K> LCDM_HD Dual<float, K> ssqrt(const Dual<float, K>& a) {
    Dual<float, K> r;
    const float rs = srsqrt(a.v);
    r.v = a.v > 0.f ? a.v * rs : sqrtf(a.v);
    const float h = 0.5f * rs;
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = a.d[k] * h;
    return r;
}
template <class T, int K> LCDM_HD Dual<T, K> sabs(const Dual<T, K>& a) { return sval(a.v) < 0 ? -a : a; }
// value with a given gradient: r = v + sum_k g_k * (tangent_k of the inputs), built by callers
template <class T, int K> LCDM_HD Dual<T, K> dlin(T v, T g, const Dual<T, K>& x) {
    Dual<T, K> r; r.v = v;
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = g * x.d[k];
    return r;
}
template <class T, int K> LCDM_HD void dacc(Dual<T, K>& r, T g, const Dual<T, K>& x) {
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = r.d[k] + g * x.d[k];
}
template <class T, int K> struct CstImpl<Dual<T, K> > {
    static LCDM_HD Dual<T, K> make(double v) { return dconst<T, K>(CstImpl<T>::make(v)); }
};
// base scalar of a (possibly dual) scalar, and constants of that base type
template <class S> struct Base { typedef S type; };
template <class T, int K> struct Base<Dual<T, K> > { typedef T type; };
template <class S> LCDM_HD typename Base<S>::type cst_like(const S&, double v) {
    return cst<typename Base<S>::type>(v);
}
// plain scalars behave as duals with no tangent
LCDM_HD float vof(float a) { return a; }
LCDM_HD double vof(double a) { return a; }
template <class T, int K> LCDM_HD T vof(const Dual<T, K>& a) { return a.v; }

// ---------------------------------------------------------------------------
// Complex numbers over scalar S (S = T or Dual<T,K>)
// ---------------------------------------------------------------------------
template <class S>
struct Cx {
    S re, im;
};
template <class S> LCDM_HD Cx<S> mkcx(const S& r, const S& i) { Cx<S> c; c.re = r; c.im = i; return c; }
template <class S> LCDM_HD Cx<S> operator+(const Cx<S>& a, const Cx<S>& b) { return mkcx<S>(a.re + b.re, a.im + b.im); }
template <class S> LCDM_HD Cx<S> operator-(const Cx<S>& a, const Cx<S>& b) { return mkcx<S>(a.re - b.re, a.im - b.im); }
template <class S> LCDM_HD Cx<S> operator-(const Cx<S>& a) { return mkcx<S>(-a.re, -a.im); }
template <class S> LCDM_HD Cx<S> operator*(const Cx<S>& a, const Cx<S>& b) {
    return mkcx<S>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class S> LCDM_HD Cx<S> operator/(const Cx<S>& a, const Cx<S>& b) {
    S n = b.re * b.re + b.im * b.im;
    return mkcx<S>((a.re * b.re + a.im * b.im) / n, (a.im * b.re - a.re * b.im) / n);
}
template <class S, class R> LCDM_HD Cx<S> cxadd(const Cx<S>& a, const R& s) { return mkcx<S>(a.re + s, a.im); }
template <class S, class R> LCDM_HD Cx<S> cxrsub(const R& s, const Cx<S>& a) { return mkcx<S>(s - a.re, -a.im); }
template <class S, class R> LCDM_HD Cx<S> cxscale(const Cx<S>& a, const R& s) { return mkcx<S>(a.re * s, a.im * s); }
template <class S> LCDM_HD Cx<S> conj(const Cx<S>& a) { return mkcx<S>(a.re, -a.im); }
template <class S> LCDM_HD S norm2(const Cx<S>& a) { return a.re * a.re + a.im * a.im; }
template <class S> LCDM_HD Cx<S> cxrcp(const Cx<S>& a) {
    S n = a.re * a.re + a.im * a.im;
    S in = cst_like(n, 1.0) / n;
    return mkcx<S>(a.re * in, -(a.im * in));
}
// principal square root
template <class S> LCDM_HD Cx<S> cxsqrt(const Cx<S>& a) {
    S r = ssqrt(a.re * a.re + a.im * a.im);
    bool neg_im = sval(vof(a.im)) < 0;
    if (sval(vof(a.re)) >= 0) {
        S t = ssqrt((r + a.re) * cst_like(r, 0.5));
        return mkcx<S>(t, a.im / (t + t));
    }
    S t = ssqrt((r - a.re) * cst_like(r, 0.5));
    S ai = neg_im ? -a.im : a.im;
    return mkcx<S>(ai / (t + t), neg_im ? -t : t);
}

// With tangents: the value by the plain complex square root, the tangents as
// d sqrt(a) = da / (2 sqrt(a)) with one complex reciprocal for all of them.
template <class T, int K> LCDM_HD Cx<Dual<T, K> > cxsqrt(const Cx<Dual<T, K> >& a) {
    const Cx<T> sv = cxsqrt(mkcx<T>(a.re.v, a.im.v));
    const T h = cst<T>(0.5) / (sv.re * sv.re + sv.im * sv.im);
    const T cr = sv.re * h, ci = -(sv.im * h);      // 1 / (2 sqrt(a))
    Cx<Dual<T, K> > r;
    r.re.v = sv.re;
    r.im.v = sv.im;
#pragma unroll
    for (int k = 0; k < K; k++) {
        r.re.d[k] = a.re.d[k] * cr - a.im.d[k] * ci;
        r.im.d[k] = a.re.d[k] * ci + a.im.d[k] * cr;
    }
    return r;
}

// ---------------------------------------------------------------------------
// Root / argument pairs.  A pair is two numbers that are either complex
// conjugates (CPair, stores the first member) or two reals (RPair).
// ---------------------------------------------------------------------------
template <class S> struct CPair { Cx<S> c; };
template <class S> struct RPair { S a, b; };

template <class S> LCDM_HD CPair<S> mkcp(const Cx<S>& c) { CPair<S> p; p.c = c; return p; }
template <class S> LCDM_HD RPair<S> mkrp(const S& a, const S& b) { RPair<S> p; p.a = a; p.b = b; return p; }

// sum and product of the two members (real in both cases)
template <class S> LCDM_HD S psum(const CPair<S>& p) { return p.c.re + p.c.re; }
template <class S> LCDM_HD S psum(const RPair<S>& p) { return p.a + p.b; }
template <class S> LCDM_HD S pprod(const CPair<S>& p) { return norm2(p.c); }
template <class S> LCDM_HD S pprod(const RPair<S>& p) { return p.a * p.b; }
// exchange the members
template <class S> LCDM_HD CPair<S> pswap(const CPair<S>& p) { return mkcp(conj(p.c)); }
template <class S> LCDM_HD RPair<S> pswap(const RPair<S>& p) { return mkrp(p.b, p.a); }
// member-wise arithmetic
template <class S> LCDM_HD CPair<S> operator+(const CPair<S>& p, const CPair<S>& q) { return mkcp(p.c + q.c); }
template <class S> LCDM_HD RPair<S> operator+(const RPair<S>& p, const RPair<S>& q) { return mkrp(p.a + q.a, p.b + q.b); }
template <class S> LCDM_HD CPair<S> operator-(const CPair<S>& p, const CPair<S>& q) { return mkcp(p.c - q.c); }
template <class S> LCDM_HD RPair<S> operator-(const RPair<S>& p, const RPair<S>& q) { return mkrp(p.a - q.a, p.b - q.b); }
template <class S> LCDM_HD CPair<S> operator*(const CPair<S>& p, const CPair<S>& q) { return mkcp(p.c * q.c); }
template <class S> LCDM_HD RPair<S> operator*(const RPair<S>& p, const RPair<S>& q) { return mkrp(p.a * q.a, p.b * q.b); }
template <class S> LCDM_HD CPair<S> operator/(const CPair<S>& p, const CPair<S>& q) { return mkcp(p.c / q.c); }
template <class S> LCDM_HD RPair<S> operator/(const RPair<S>& p, const RPair<S>& q) { return mkrp(p.a / q.a, p.b / q.b); }
template <class S, class R> LCDM_HD CPair<S> padd(const CPair<S>& p, const R& s) { return mkcp(cxadd(p.c, s)); }
template <class S, class R> LCDM_HD RPair<S> padd(const RPair<S>& p, const R& s) { return mkrp<S>(p.a + s, p.b + s); }
template <class S, class R> LCDM_HD CPair<S> prsub(const R& s, const CPair<S>& p) { return mkcp(cxrsub(s, p.c)); }
template <class S, class R> LCDM_HD RPair<S> prsub(const R& s, const RPair<S>& p) { return mkrp<S>(s - p.a, s - p.b); }
template <class S, class R> LCDM_HD CPair<S> pscale(const CPair<S>& p, const R& s) { return mkcp(cxscale(p.c, s)); }
template <class S, class R> LCDM_HD RPair<S> pscale(const RPair<S>& p, const R& s) { return mkrp<S>(p.a * s, p.b * s); }
template <class S> LCDM_HD CPair<S> psqrt(const CPair<S>& p) { return mkcp(cxsqrt(p.c)); }
template <class S> LCDM_HD RPair<S> psqrt(const RPair<S>& p) { return mkrp(ssqrt(p.a), ssqrt(p.b)); }
template <class S> LCDM_HD CPair<S> prcp(const CPair<S>& p) { return mkcp(cxrcp(p.c)); }
template <class S> LCDM_HD RPair<S> prcp(const RPair<S>& p) {
    return mkrp<S>(cst_like(p.a, 1.0) / p.a, cst_like(p.b, 1.0) / p.b);
}
// sum over members of c_m * x_m (real)
template <class T> LCDM_HD T pdot(const CPair<T>& c, const CPair<T>& x) {
    return cst<T>(2.0) * (c.c.re * x.c.re - c.c.im * x.c.im);
}
template <class T> LCDM_HD T pdot(const RPair<T>& c, const RPair<T>& x) { return c.a * x.a + c.b * x.b; }
// values of a dual pair
template <class T, int K> LCDM_HD CPair<T> pval(const CPair<Dual<T, K> >& p) { return mkcp(mkcx<T>(p.c.re.v, p.c.im.v)); }
template <class T, int K> LCDM_HD RPair<T> pval(const RPair<Dual<T, K> >& p) { return mkrp<T>(p.a.v, p.b.v); }
template <class T> LCDM_HD CPair<T> pval(const CPair<T>& p) { return p; }
template <class T> LCDM_HD RPair<T> pval(const RPair<T>& p) { return p; }
// ---------------------------------------------------------------------------
// Carlson's duplication algorithm (ref. [10]).
// Deviation tolerance: the iteration stops once every argument is within
// tol * mean of the common mean; the truncated series is then exact to
// about c tol^6, where c is small (the omitted degree-6 terms have
// coefficients of a few hundredths and E2 is itself O(tol^2)).  FP32: 0.10,
// at which the outputs' largest errors on the benchmark and stress draws are
// those of 0.06 and the sequence takes 0.37 fewer steps per pair; FP64:
// 1.5e-3.
// ---------------------------------------------------------------------------
template <class T> struct Prec;
template <> struct Prec<float> {
    static LCDM_HD float tol() { return 0.10f; }
    static LCDM_HD float rc_series_max() { return 0.1f; }
    enum { rc_terms = 6, maxit = 24 };
};
template <> struct Prec<double> {
    static LCDM_HD double tol() { return 1.5e-3; }
    static LCDM_HD double rc_series_max() { return 0.03; }
    enum { rc_terms = 12, maxit = 40 };
};

// dual numbers follow the precision of their base type
template <class T, int K> struct Prec<Dual<T, K> > {
    static LCDM_HD Dual<T, K> tol() { return dconst<T, K>(Prec<T>::tol()); }
    static LCDM_HD Dual<T, K> rc_series_max() { return dconst<T, K>(Prec<T>::rc_series_max()); }
    enum { rc_terms = Prec<T>::rc_terms, maxit = Prec<T>::maxit };
};

// R_C(x, y) = R_F(x, y, y) (eq. 2.8) by duplication; value only.
template <class T> LCDM_NI T rc_value(T x, T y, int* fail) {
    const T tol = Prec<T>::tol();
    int m = 0;
    T A = (x + y + y) * cst<T>(1.0 / 3.0);
#pragma unroll 1
    for (; m < Prec<T>::maxit; m++) {
        T dv = sabs(y - A);
        if (sval(dv) <= sval(tol * sabs(A))) break;
        T lam = cst<T>(2.0) * ssqrt(x) * ssqrt(y) + y;
        x = (x + lam) * cst<T>(0.25);
        y = (y + lam) * cst<T>(0.25);
        A = (x + y + y) * cst<T>(1.0 / 3.0);
    }
    if (m == Prec<T>::maxit) *fail = 1;
    T s = (y - A) / A;
    T ser = cst<T>(159.0 / 208.0) + s * cst<T>(9.0 / 8.0);
    ser = cst<T>(9.0 / 22.0) + s * ser;
    ser = cst<T>(3.0 / 8.0) + s * ser;
    ser = cst<T>(1.0 / 7.0) + s * ser;
    ser = cst<T>(3.0 / 10.0) + s * ser;
    ser = cst<T>(1.0) + s * s * ser;
    return ser / ssqrt(A);
}

// R_C(1, 1 + e) for |e| < 1: sum_n (-e)^n / (2n+1) when e is small, else duplication.
template <class T> LCDM_HD T rc1(T e, int* fail) {
    if (sval(sabs(e)) <= sval(Prec<T>::rc_series_max())) {
        T w = -e;
        T s = cst<T>(1.0 / (2 * Prec<T>::rc_terms + 1));
#pragma unroll
        for (int n = Prec<T>::rc_terms - 1; n >= 0; n--) s = cst<T>(1.0 / (2 * n + 1)) + w * s;
        return s;
    }
    return rc_value(cst<T>(1.0), cst<T>(1.0) + e, fail);
}

// With tangents: the series and its derivative by one Horner pass in plain
// arithmetic, applied to e's tangents once (d R_C(1, 1+e)/de = -s'(w), w = -e).
template <class T, int K> LCDM_HD Dual<T, K> rc1(const Dual<T, K>& e, int* fail) {
    if (sval(sabs(e.v)) <= sval(Prec<T>::rc_series_max())) {
        const T w = -e.v;
        T s = cst<T>(1.0 / (2 * Prec<T>::rc_terms + 1)), ds = cst<T>(0.0);
#pragma unroll
        for (int n = Prec<T>::rc_terms - 1; n >= 0; n--) {
            ds = ds * w + s;
            s = cst<T>(1.0 / (2 * n + 1)) + w * s;
        }
        Dual<T, K> r;
        r.v = s;
#pragma unroll
        for (int k = 0; k < K; k++) r.d[k] = -ds * e.d[k];
        return r;
    }
    return rc_value(dconst<T, K>(cst<T>(1.0)), dconst<T, K>(cst<T>(1.0)) + e, fail);
}

// (R_C(1, 1+e) - 1) / e = sum_{n>=1} (-e)^n / (2n+1) / e, without cancellation.
template <class T> LCDM_HD T rc1_minus1_over_e(T e, int* fail) {
    if (sval(sabs(e)) <= sval(Prec<T>::rc_series_max())) {
        T w = -e;
        T s = cst<T>(-1.0 / (2 * Prec<T>::rc_terms + 3));
#pragma unroll
        for (int n = Prec<T>::rc_terms; n >= 1; n--) s = cst<T>(-1.0 / (2 * n + 1)) + w * s;
        return s;
    }
    return (rc_value(cst<T>(1.0), cst<T>(1.0) + e, fail) - cst<T>(1.0)) / e;
}

// Series of R_J (and of R_D = R_J with p equal to one argument) in the
// normalised deviations: X for the single argument, sumY / prodY for the pair,
// P for p.  U is a scalar or a complex type.
template <class U, class T> LCDM_HD U rj_series(U X, U sumY, U prodY, U P) {
    U XYZ = X * prodY;
    U P2 = P * P;
    U E2 = X * sumY + prodY - P2 * cst<T>(3.0);
    U E3 = XYZ + E2 * P * cst<T>(2.0) + P2 * P * cst<T>(4.0);
    U E4 = (XYZ * cst<T>(2.0) + E2 * P + P2 * P * cst<T>(3.0)) * P;
    U E5 = XYZ * P2;
    return cst<T>(1.0) - E2 * cst<T>(3.0 / 14.0) + E3 * cst<T>(1.0 / 6.0) + E2 * E2 * cst<T>(9.0 / 88.0)
           - E4 * cst<T>(3.0 / 22.0) - E2 * E3 * cst<T>(9.0 / 52.0) + E5 * cst<T>(3.0 / 26.0);
}

// The R_F and R_J series of the duplication's last step, as plain numbers or
// with tangents.  For dual numbers the series' partial derivatives with
// respect to its four inputs are formed by hand (reverse mode through the
// polynomial, in plain arithmetic) and applied to the inputs' tangents once:
// a fraction of the cost of carrying K tangents through every product.
//   R_F: 1 - e2/10 + e3/14 + e2^2/24 - 3 e2 e3/44,  e2 = X sY + pY, e3 = X pY.
template <class S> LCDM_HD S rf_ser(const S& X, const S& sY, const S& pY) {
    typedef typename Base<S>::type T;
    S e2 = X * sY + pY, e3 = X * pY;
    return cst<T>(1.0) - e2 * cst<T>(0.1) + e3 * cst<T>(1.0 / 14.0) + e2 * e2 * cst<T>(1.0 / 24.0)
           - e2 * e3 * cst<T>(3.0 / 44.0);
}
template <class T, int K> LCDM_HD Dual<T, K> rf_ser(const Dual<T, K>& X, const Dual<T, K>& sY, const Dual<T, K>& pY) {
    const T x = X.v, sy = sY.v, py = pY.v;
    const T e2 = x * sy + py, e3 = x * py;
    Dual<T, K> r;
    r.v = cst<T>(1.0) - e2 * cst<T>(0.1) + e3 * cst<T>(1.0 / 14.0) + e2 * e2 * cst<T>(1.0 / 24.0)
          - e2 * e3 * cst<T>(3.0 / 44.0);
    const T g2 = cst<T>(-0.1) + e2 * cst<T>(1.0 / 12.0) - e3 * cst<T>(3.0 / 44.0);
    const T g3 = cst<T>(1.0 / 14.0) - e2 * cst<T>(3.0 / 44.0);
    const T gx = g2 * sy + g3 * py, gs = g2 * x, gp = g2 + g3 * x;
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = gx * X.d[k] + gs * sY.d[k] + gp * pY.d[k];
    return r;
}
//   R_J (rj_series above): Q = X pY, E2 = X sY + pY - 3P^2, E3 = Q + 2 E2 P + 4 P^3,
//   E4 = (2Q + E2 P + 3P^3) P, E5 = Q P^2.
template <class S> LCDM_HD S rj_ser(const S& X, const S& sY, const S& pY, const S& P) {
    return rj_series<S, typename Base<S>::type>(X, sY, pY, P);
}
template <class T, int K>
LCDM_HD Dual<T, K> rj_ser(const Dual<T, K>& X, const Dual<T, K>& sY, const Dual<T, K>& pY, const Dual<T, K>& P) {
    const T x = X.v, sy = sY.v, py = pY.v, p = P.v;
    const T Q = x * py, P2 = p * p, P3 = P2 * p;
    const T E2 = x * sy + py - P2 * cst<T>(3.0);
    const T E3 = Q + E2 * p * cst<T>(2.0) + P3 * cst<T>(4.0);
    const T W = Q * cst<T>(2.0) + E2 * p + P3 * cst<T>(3.0);
    const T E4 = W * p, E5 = Q * P2;
    Dual<T, K> r;
    r.v = cst<T>(1.0) - E2 * cst<T>(3.0 / 14.0) + E3 * cst<T>(1.0 / 6.0) + E2 * E2 * cst<T>(9.0 / 88.0)
          - E4 * cst<T>(3.0 / 22.0) - E2 * E3 * cst<T>(9.0 / 52.0) + E5 * cst<T>(3.0 / 26.0);
    // adjoints of the intermediates (d series / d E_i), then back to the inputs
    const T gE3 = cst<T>(1.0 / 6.0) - E2 * cst<T>(9.0 / 52.0);
    const T gE4 = cst<T>(-3.0 / 22.0), gE5 = cst<T>(3.0 / 26.0);
    const T gW = gE4 * p;
    const T gE2 = cst<T>(-3.0 / 14.0) + E2 * cst<T>(9.0 / 44.0) - E3 * cst<T>(9.0 / 52.0) + gW * p
                  + gE3 * p * cst<T>(2.0);
    const T gQ = gE5 * P2 + gW * cst<T>(2.0) + gE3;
    const T gP3 = gW * cst<T>(3.0) + gE3 * cst<T>(4.0);
    const T gP2 = gE5 * Q - gE2 * cst<T>(3.0) + gP3 * p;
    const T gp = gE4 * W + gW * E2 + gE3 * E2 * cst<T>(2.0) + gP3 * P2 + gP2 * p * cst<T>(2.0);
    const T gx = gE2 * sy + gQ * py, gs = gE2 * x, gy = gE2 + gQ * x;
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = gx * X.d[k] + gs * sY.d[k] + gy * pY.d[k] + gp * P.d[k];
    return r;
}

// Divided-difference numbers: the values of a quantity at two points u1, u2
// and its divided difference (v1 - v2) / (u1 - u2), with the product rule
// [fg] = [f] g(u1) + f(u2) [g].  Used to evaluate R_J(p) - R_J(p') for close
// p, p' without cancellation.
template <class T> struct DD { T v1, v2, d; };
template <class T> LCDM_HD DD<T> mkdd(T a, T b, T d) { DD<T> r; r.v1 = a; r.v2 = b; r.d = d; return r; }
template <class T> LCDM_HD DD<T> operator+(const DD<T>& a, const DD<T>& b) { return mkdd<T>(a.v1 + b.v1, a.v2 + b.v2, a.d + b.d); }
template <class T> LCDM_HD DD<T> operator-(const DD<T>& a, const DD<T>& b) { return mkdd<T>(a.v1 - b.v1, a.v2 - b.v2, a.d - b.d); }
template <class T> LCDM_HD DD<T> operator*(const DD<T>& a, const DD<T>& b) {
    return mkdd<T>(a.v1 * b.v1, a.v2 * b.v2, a.d * b.v1 + a.v2 * b.d);
}
template <class T> LCDM_HD DD<T> operator*(const DD<T>& a, const T& c) { return mkdd<T>(a.v1 * c, a.v2 * c, a.d * c); }
template <class T> LCDM_HD DD<T> operator+(const DD<T>& a, const T& c) { return mkdd<T>(a.v1 + c, a.v2 + c, a.d); }
template <class T> LCDM_HD DD<T> operator-(const T& c, const DD<T>& a) { return mkdd<T>(c - a.v1, c - a.v2, -a.d); }
template <class T> LCDM_HD DD<T> operator-(const DD<T>& a, const T& c) { return mkdd<T>(a.v1 - c, a.v2 - c, a.d); }

// Even exponent of the largest argument (0 for zero, subnormal or non-finite
// magnitudes), read from the float's exponent bits.
LCDM_HD int even_exponent(float mag) {
    uint32_t b;
    memcpy(&b, &mag, sizeof b);
    const int be = (int)((b >> 23) & 0xffu);
    const int e = (be == 0 || be == 0xff) ? 0 : be - 127;
    return e & ~1;
}

// 2^k exactly, from its bit pattern (|k| <= 126: a normal number in either
// precision).  Multiplying by it is exact and, unlike ldexp, one instruction.
template <class B> LCDM_HD B pow2i(int k);
template <> LCDM_HD float pow2i<float>(int k) {
    const uint32_t b = (uint32_t)(k + 127) << 23;
    float f;
    memcpy(&f, &b, sizeof f);
    return f;
}
template <> LCDM_HD double pow2i<double>(int k) {
    const uint64_t b = (uint64_t)(k + 1023) << 52;
    double f;
    memcpy(&f, &b, sizeof f);
    return f;
}

// ---------------------------------------------------------------------------
// The same duplication sequence for R_F(x1, y_a, y_b), R_D(y_a, y_b, x1) and
// NJ R_J(x1, y_a, y_b, p_j) (and the divided-difference track), all symmetric
// in the pair (y_a, y_b), carried on real numbers only: the pair enters
// through sigma = y_a + y_b and pi = y_a y_b, and its square roots through
// S = s_a + s_b and P = s_a s_b (real for a conjugate pair as for two reals).
// One step, with s1 = sqrt(x1), lambda = s1 S + P:
//   x1 + lambda = (s1 + s_a)(s1 + s_b) = s1^2 + s1 S + P,
//   sigma' = S (S + 2 s1) / 4,   pi' = x1' S^2 / 4,   x1' = (x1 + lambda) / 4
// (y_a + lambda = (s_a + s1)(s_a + s_b)): sums and products of non-negative
// numbers, so no step cancels, not even for a pair near the negative real
// axis.  The square roots of the starting triple are given (u1 and the pair
// u of the callers, x1 = u1^2, y = u^2), so the first step takes none; after
// it the pair lies in the right half-plane and P = sqrt(pi),
// S = sqrt(sigma + 2P) add positive numbers.  For the stopping rule the
// pair's distance from the mean mu follows from
//   (y_a - mu)(y_b - mu) = pi - mu sigma + mu^2   (|y - mu|^2 for a conjugate pair),
//   (y_a - mu)^2 + (y_b - mu)^2 = (sigma - 2 mu)^2 - 2 (pi - mu sigma + mu^2)   (two reals).
// The caller gives, per track, delta_j = (p_j - x1)(p_j - y_a)(p_j - y_b)
// (formed from the members, where it does not cancel) and, for the
// divided-difference track, hl = p_last - x1 and PiL = (p_last - y_a)(p_last - y_b).
// ---------------------------------------------------------------------------
template <class T, int NJ>
struct SymResult {
    T RF;      // R_F(x1, y_a, y_b)
    T RD1;     // R_D(y_a, y_b, x1)
    T RJ[NJ > 0 ? NJ : 1];
    T DJ;      // (R_J(last track) - R_D1) / hl   (DDL)
};

template <class T, int NJ, bool WANT_D, bool DDL = false>
LCDM_HD SymResult<T, NJ> carlson_sym(T s1, T S, T P, bool cplx, const T* pj, const T* dj, int* fail, T hl = T(),
                                     T PiL = T()) {
    static_assert(!DDL || (WANT_D && NJ > 0), "the divided-difference track needs R_D and an R_J track");
    SymResult<T, NJ> R;
    float mag = fabsf((float)sval(s1));
    mag = mag * mag;
    {
        const float a = fabsf((float)sval(S)), b = fabsf((float)sval(P));
        if (a * a > mag) mag = a * a;
        if (b > mag) mag = b;
    }
    T p[NJ > 0 ? NJ : 1], delta[NJ > 0 ? NJ : 1], sJ[NJ > 0 ? NJ : 1];
#pragma unroll
    for (int j = 0; j < NJ; j++) {
        p[j] = pj[j];
        const float a = fabsf((float)sval(p[j]));
        if (a > mag) mag = a;
    }
    // scale by 2^-e, e even: x, y, p by g = 2^-e, square roots by h = 2^-e/2;
    // the results scale back by h (R_F) and h g (R_D, R_J), h g g (DJ), one
    // factor at a time so that every factor is a normal number
    typedef typename Base<T>::type BT;
    int e = even_exponent(mag);
    e = e > 124 ? 124 : (e < -124 ? -124 : e);
    const BT h = pow2i<BT>(-e / 2), g = pow2i<BT>(-e);
    s1 = s1 * h;
    S = S * h;
    P = P * g;
    T x1 = s1 * s1;
    T sig = S * S - cst<T>(2.0) * P;   // exact enough for the first stopping test (see above)
    T pi = P * P;
#pragma unroll
    for (int j = 0; j < NJ; j++) {
        p[j] = p[j] * g;
        delta[j] = dj[j] * g * g * g;
        sJ[j] = cst<T>(0.0);
    }
    T sD1 = cst<T>(0.0);
    T f = cst<T>(1.0);
    T hs = cst<T>(0.0), sDD = cst<T>(0.0);
    if (DDL) {
        hs = hl * g;
        PiL = PiL * g * g;
    }
    const T tol = Prec<T>::tol();
    int m = 0;
#pragma unroll 1
    for (; m < Prec<T>::maxit; m++) {
        T mu = x1 + sig;
#pragma unroll
        for (int j = 0; j < NJ; j++) mu = mu + p[j];
        mu = mu * cst<T>(1.0 / (3 + NJ));
        T lim = tol * mu;
        T lim2 = lim * lim;
        T dx = x1 - mu;
        T v = pi - mu * sig + mu * mu;
        T u = sig - cst<T>(2.0) * mu;
        T dev2 = cplx ? v : u * u - cst<T>(2.0) * v;
        bool conv = sval(dx * dx) <= sval(lim2) && sval(dev2) <= sval(lim2);
#pragma unroll
        for (int j = 0; j < NJ; j++) {
            T dp = p[j] - mu;
            conv = conv && sval(dp * dp) <= sval(lim2);
        }
        if (conv) break;
        if (m > 0) {
            s1 = ssqrt(x1);
            P = ssqrt(pi);
            S = ssqrt(sig + cst<T>(2.0) * P);
        }
        T lam = s1 * S + P;
        T xl = x1 + lam;                       // (s1 + s_a)(s1 + s_b)
        if (WANT_D) sD1 = sD1 + f / (s1 * xl);
#pragma unroll
        for (int j = 0; j < NJ; j++) {
            T sq = ssqrt(p[j]);
            T g = p[j] + sq * S + P;           // (sq + s_a)(sq + s_b)
            T d = (sq + s1) * g;
            T f3 = f * f * f;
            T ee = f3 * delta[j] / (d * d);
            if (!(DDL && j == NJ - 1)) sJ[j] = sJ[j] + f * rc1(ee, fail) / d;
            if (DDL && j == NJ - 1) {
                // [R_C(1,1+e)/d_p - 1/d_x1] / h with e/h = f^3 Pi / d_p^2 and
                // (d_p - d_x1)/h = f [g(a) + 2b (a + b + S)] / (a + b),
                // a = sqrt(p), b = s1, g(v) = (v + s_a)(v + s_b), d_x1 = 2 b g(b),
                // g(b) = x1 + lambda
                T eh = f3 * PiL / (d * d);
                T F1 = rc1_minus1_over_e(ee, fail);
                T dx1 = cst<T>(2.0) * s1 * xl;
                T ddp = f * (g + cst<T>(2.0) * s1 * (sq + s1 + S)) / (sq + s1);
                sDD = sDD + f * (eh * F1 / d - ddp / (d * dx1));
            }
        }
        x1 = xl * cst<T>(0.25);
        sig = S * (S + cst<T>(2.0) * s1) * cst<T>(0.25);
        pi = x1 * (S * S) * cst<T>(0.25);
#pragma unroll
        for (int j = 0; j < NJ; j++) p[j] = (p[j] + lam) * cst<T>(0.25);
        f = f * cst<T>(0.25);
    }
    if (m == Prec<T>::maxit) *fail = 1;
    // R_F series: Y_a + Y_b = (2A - sigma)/A, Y_a Y_b = (A^2 - A sigma + pi)/A^2
    {
        T A = (x1 + sig) * cst<T>(1.0 / 3.0), iA = cst<T>(1.0) / A;
        T X = (A - x1) * iA;
        T sY = (A + A - sig) * iA, pY = ((A - sig) * A + pi) * (iA * iA);
        T ser = rf_ser(X, sY, pY);
        R.RF = ser / ssqrt(A) * h;
    }
    if (WANT_D) {
        T A = (sig + cst<T>(3.0) * x1) * cst<T>(0.2), iA = cst<T>(1.0) / A;
        T X = (A - x1) * iA;
        T sY = (A + A - sig) * iA, pY = ((A - sig) * A + pi) * (iA * iA);
        T ser = rj_ser(X, sY, pY, X);
        R.RD1 = (f * ser * iA / ssqrt(A) + cst<T>(3.0) * sD1) * g * h;
    } else {
        R.RD1 = R.RF;
    }
#pragma unroll
    for (int j = 0; j < (DDL ? NJ - 1 : NJ); j++) {
        T A = (x1 + sig + cst<T>(2.0) * p[j]) * cst<T>(0.2), iA = cst<T>(1.0) / A;
        T X = (A - x1) * iA, Pp = (A - p[j]) * iA;
        T sY = (A + A - sig) * iA, pY = ((A - sig) * A + pi) * (iA * iA);
        T ser = rj_ser(X, sY, pY, Pp);
        R.RJ[j] = (f * ser * iA / ssqrt(A) + cst<T>(6.0) * sJ[j]) * g * h;
    }
    R.DJ = R.RD1;
    if (DDL) {
        // final series: A(u) = (sig + 2u)/5 at u1 = p, u2 = x1; X = 1 - x1/A,
        // Y = 1 - pair/A, P = 1 - u/A; divided differences by the product rule,
        // [A^-3/2] = -(2/5)(A1 + sqrt(A1 A2) + A2) / ((sqrt A1 + sqrt A2) A1^3/2 A2^3/2);
        // R_J(p) - R_D = f (T(u1) - T(u2)) + 6 (sum_p - sum_x1), T = A^-3/2 S
        const T sgm = x1 + sig;
        const T u1 = x1 + hs * f;
        T A1 = (sgm + cst<T>(2.0) * u1) * cst<T>(0.2), A2 = (sgm + cst<T>(2.0) * x1) * cst<T>(0.2);
        T iA1 = cst<T>(1.0) / A1, iA2 = cst<T>(1.0) / A2;
        T dInv = cst<T>(-0.4) * iA1 * iA2;
        DD<T> inv = mkdd<T>(iA1, iA2, dInv);
        DD<T> X = cst<T>(1.0) - inv * x1;
        DD<T> sY = cst<T>(2.0) - inv * sig;
        DD<T> inv2 = inv * inv;
        DD<T> pY = (cst<T>(1.0) - inv * sig) + inv2 * pi;
        DD<T> Pq = mkdd<T>(cst<T>(1.0) - u1 * iA1, cst<T>(1.0) - x1 * iA2, sgm * cst<T>(-0.2) * iA1 * iA2);
        DD<T> ser = rj_series<DD<T>, T>(X, sY, pY, Pq);
        T r1 = ssqrt(A1), r2 = ssqrt(A2);
        T a32_1 = iA1 / r1, a32_2 = iA2 / r2;
        T dA32 = cst<T>(-0.4) * (A1 + r1 * r2 + A2) / (r1 + r2) * a32_1 * a32_2;
        T dser = dA32 * ser.v1 + a32_2 * ser.d;
        R.DJ = (f * f * dser + cst<T>(6.0) * sDD) * g * g * h;
        R.RJ[NJ - 1] = R.RD1 + hl * R.DJ;
    }
    return R;
}

// Square roots' sum S and product P of the pair whose members are the squares
// of u (the callers' u's: y = u^2, principal roots |u| resp. +-u with Re >= 0).
template <class S> LCDM_HD S proot_sum(const CPair<S>& u) { return sabs(u.c.re) * cst_like(u.c.re, 2.0); }
template <class S> LCDM_HD S proot_sum(const RPair<S>& u) { return sabs(u.a) + sabs(u.b); }
template <class S> LCDM_HD S proot_prod(const CPair<S>& u) { return norm2(u.c); }
template <class S> LCDM_HD S proot_prod(const RPair<S>& u) { return sabs(u.a * u.b); }
template <class S> LCDM_HD bool pis_cplx(const CPair<S>&) { return true; }
template <class S> LCDM_HD bool pis_cplx(const RPair<S>&) { return false; }

}  // namespace lcdm
