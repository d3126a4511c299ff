// Kernels of the distance path:
//   (the root preparation kernel is in lcdm_prep.cuh)
//   pairs_kernel  persistent warps over contiguous ranges of (cosmology,
//                 redshift) pairs: distance integrals (3.7)-(3.9) / (B.1)-(B.3),
//                 observables, tangents, and the per-cosmology reductions of the
//                 vector-Jacobian product and of the Gaussian log-likelihood.
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include <type_traits>

#include "lcdm_dist.cuh"

namespace lcdm {

// Physical constants: speed of light [km/s]; Hubble time unit: 1 Mpc/km in Gyr.
#define LCDM_C_KMS 299792.458
#define LCDM_HUBBLE_GYR 977.7922216807891

// ----------------------------------------------------------------------------
// Per-cosmology record (FP64 master; a hi/lo float copy for the mixed path).
// Roots are in z (r = rho - 1).  kind: 0 quartic, two real roots + conjugate
// pair; 1 quartic, four real; 2 cubic, one real + pair; 3 cubic, three real.
// For kinds 0/2 (P_re, P_im) is the pair member with positive imaginary part;
// for kinds 1/3 they are the two real members.
// ----------------------------------------------------------------------------
enum RecField {
    RF_A = 0, RF_B, RF_PRE, RF_PIM, RF_YA, RF_YB, RF_YPRE, RF_YPIM,
    RF_AMH, RF_OK, RF_H0, RF_DH, RF_TH, RF_KIND,
    // quartic big-root quantities: lam = Or, a_A = -lam A, m_A = lam rho_A, eps_A = -1/rho_A, rho_A
    RF_LAM, RF_AA, RF_MA, RF_EPSA, RF_RHOA,
    // tangents (RF_KT slots each: Om, OL, Or, Ok, Os, Ox; the first ncol - 1 used)
    RF_DA = 19, RF_DB = 25, RF_DPRE = 31, RF_DPIM = 37, RF_DAMH = 43, RF_DOK = 49,
    RF_DLAM = 55, RF_DAA = 61, RF_DMA = 67, RF_DEPSA = 73, RF_DRHOA = 79,
    // q_j = -1/r_j for A, B and the pair (the two real members for kinds 1/3),
    // and the scale N = sqrt(E^2(0) / alpha_n) of the Carlson arguments
    RF_QA = 85, RF_QB, RF_QPRE, RF_QPIM, RF_NRM,
    RF_DQA = 90, RF_DQB = 96, RF_DQPRE = 102, RF_DQPIM = 108, RF_DNRM = 114,
    NREC = 120
};
enum { RF_KT = 6 };   // tangent slots per field: at most six density directions

enum CosmoStatus {
    ST_OK = 0, ST_NO_BIG_BANG = 1, ST_INVALID = 2, ST_DEGENERATE = 3, ST_NOCONV = 4, ST_UNSUPPORTED = 5
};

// ------------------------------------------------------------ observables ---
LCDM_HD float expm1_(float x) { return expm1f(x); }
LCDM_HD double expm1_(double x) { return expm1(x); }
LCDM_HD void sincos_(float x, float* s, float* c) { sincosf(x, s, c); }
LCDM_HD void sincos_(double x, double* s, double* c) { sincos(x, s, c); }

// S_k(D): sinh / sin form, or its Taylor series in u = Ok D^2 near flatness,
// with dS/dD and dS/dOk ([59] eqs. 13.47, 13.57 as cited in Sec. 2.1.1).
template <class T> LCDM_HD void curv_map(T D, T Ok, T& S, T& SD, T& Sk) {
    T u = Ok * D * D;
    if (fabs(u) < (T)0.05) {
        // coefficients 1/(2n+1)!, 1/(2n)!
        constexpr double cs[8] = {1.0, 1.0 / 6, 1.0 / 120, 1.0 / 5040, 1.0 / 362880, 1.0 / 39916800,
                                  1.0 / 6227020800.0, 1.0 / 1307674368000.0};
        constexpr double cd2[8] = {1.0, 0.5, 1.0 / 24, 1.0 / 720, 1.0 / 40320, 1.0 / 3628800,
                                   1.0 / 479001600.0, 1.0 / 87178291200.0};
        T s = (T)cs[7], sd = (T)cd2[7], sk = (T)(7 * cs[7]);
#pragma unroll
        for (int i = 6; i >= 0; i--) {
            s = (T)cs[i] + u * s;
            sd = (T)cd2[i] + u * sd;
            if (i >= 1) sk = (T)(i * cs[i]) + u * sk;
        }
        S = D * s; SD = sd; Sk = D * D * D * sk;
        return;
    }
    if (Ok > 0) {
        // sinh and cosh from one exponential: e^x - 1 = m, sinh x = (m + m / (1 + m)) / 2
        // (both terms positive for x = sqrt(Ok) D >= 0), cosh x = ((1 + m) + 1 / (1 + m)) / 2
        T r = sqrt(Ok);
        const T m = expm1_(r * D), ex = m + (T)1;
        S = (m + m / ex) * (T)0.5 / r; SD = (ex + (T)1 / ex) * (T)0.5;
    } else {
        T r = sqrt(-Ok);
        T sn, cs;
        sincos_(r * D, &sn, &cs);
        S = sn / r; SD = cs;
    }
    Sk = (D * SD - S) / (2 * Ok);
}

// ----------------------------------------------------------- pair kernel ----
enum Layout { LAYOUT_CSR = 0, LAYOUT_DENSE = 1, LAYOUT_SHARED = 2 };
enum Outputs { O_DC = 0, O_T = 1, O_X = 2, O_DM = 3, O_DL = 4, O_MU = 5, N_OUT = 6 };

struct PairArgs {
    const double* recD;
    const float2* recF;
    int32_t* status;
    const int64_t* offsets;
    const void* z;
    int layout;
    int64_t nrow;   // pairs per row (dense) / redshifts (shared)
    int64_t nnz;
    int64_t B;
    int ncol;
    int outmask;    // bit o: write out[o]
    void* out[N_OUT];
    void* jac[N_OUT];        // [nnz][ncol] per output, optional
    const void* cot[N_OUT];  // cotangents for the VJP, optional
    const void* mobs;        // loglike mode when non-null
    double M, sigma;
    double* grad;            // [B][ncol] accumulated (VJP or d loglike)
    double* loglike;         // [B]
    int64_t chunk;           // pairs per warp (multiple of 32)
    int64_t base;            // CSR: index of the first pair (z, outputs and offsets are absolute)
    int interleave;          // lane l takes the l-th 32nd of the warp's range (else 32 consecutive pairs)
    // deterministic reduction (optional): per warp, the partial sums of its
    // first and last rows [warp][2][RF_KT + 2] and those rows [warp][2];
    // rows owned by one warp are added directly (in program order)
    double* part;
    int64_t* wrow;
    int64_t det_cap;         // warps with slots
};
enum { DET_SLOT = RF_KT + 2 };

template <class T> struct IO;
template <> struct IO<float> { typedef float type; };
template <> struct IO<double> { typedef double type; };

// value of a record field in the pass type
template <class T> LCDM_HD T recv(const double* rd, const float2* rf, int i);
template <> LCDM_HD double recv<double>(const double* rd, const float2*, int i) { return rd[i]; }
template <> LCDM_HD float recv<float>(const double*, const float2* rf, int i) { return rf[i].x; }

// 1 + z q for a record field q.  It cancels where z q is near -1 (for the
// complex pair near z = Re r_P, which lies at z > 0 close to the no-Big-Bang
// boundary), so in FP32 q enters with its low word (hi, lo from the FP64
// record) and the sum is formed in double-float arithmetic before it is
// rounded once; FP64 rounds once by the fused multiply-add.
template <class T> LCDM_HD T one_plus_qz(const double* rd, const float2* rf, int i, T z);
template <> LCDM_HD double one_plus_qz<double>(const double* rd, const float2*, int i, double z) {
    return fma(rd[i], z, 1.0);
}
template <> LCDM_HD float one_plus_qz<float>(const double*, const float2* rf, int i, float z) {
    const float qh = rf[i].x, ql = rf[i].y;
    const float p = qh * z, e1 = fmaf(qh, z, -p);   // qh z = p + e1 exactly
    const df64 s = two_sum(1.0f, p);
    return s.hi + (s.lo + fmaf(ql, z, e1));
}

// Build the root quantities in scalar S and evaluate the integrals.
template <class T, int K, bool WT, bool WX> struct PairEval {
    typedef typename std::conditional<(K > 0), Dual<T, K>, T>::type S;
    // the integrals inline, or as one call (see quartic_integrals_call)
    static constexpr bool SPLIT = K > 3 || (K > 0 && WX);

    static LCDM_HD S val(const double* rd, const float2* rf, int i, int di) {
        S s;
        if constexpr (K > 0) {
            s.v = recv<T>(rd, rf, i);
#pragma unroll
            for (int k = 0; k < K; k++) s.d[k] = recv<T>(rd, rf, di + k);
        } else {
            s = recv<T>(rd, rf, i);
        }
        return s;
    }
    // Y = sqrt(-r) with its tangent -dr / (2Y)
    static LCDM_HD S yval(const double* rd, const float2* rf, int iy, const S& r) {
        S y;
        if constexpr (K > 0) {
            y.v = recv<T>(rd, rf, iy);
            T h = cst<T>(-0.5) / y.v;
#pragma unroll
            for (int k = 0; k < K; k++) y.d[k] = r.d[k] * h;
        } else {
            y = recv<T>(rd, rf, iy);
        }
        return y;
    }

    static LCDM_HD void run(T z, const double* rd, const float2* rf, int kind, S& Ichi,
                                               S& It, S& IX, int* fail) {
        S A = val(rd, rf, RF_A, RF_DA);
        S amh = val(rd, rf, RF_AMH, RF_DAMH);
        S YA = yval(rd, rf, RF_YA, A);
        S Pre = val(rd, rf, RF_PRE, RF_DPRE), Pim = val(rd, rf, RF_PIM, RF_DPIM);
        S qA = val(rd, rf, RF_QA, RF_DQA), nrm = val(rd, rf, RF_NRM, RF_DNRM);
        S qPre = val(rd, rf, RF_QPRE, RF_DQPRE), qPim = val(rd, rf, RF_QPIM, RF_DQPIM);
        // w_P = 1 + z q_P (its tangent z dq_P), the first member's real part
        // by one_plus_qz
        S wre = qPre * z, wim = qPim * z;
        if constexpr (K > 0) wre.v = one_plus_qz<T>(rd, rf, RF_QPRE, z);
        else wre = one_plus_qz<T>(rd, rf, RF_QPRE, z);
        if (kind == 0 || kind == 2) {
            CPair<S> P = mkcp(mkcx<S>(Pre, Pim)), wP = mkcp(mkcx<S>(wre, wim));
            Cx<S> yv;
            yv.re = val(rd, rf, RF_YPRE, RF_YPRE);
            yv.im = val(rd, rf, RF_YPIM, RF_YPIM);
            if constexpr (K > 0) {
                // dY = -dP / (2Y), complex
                Cx<T> y0 = mkcx<T>(yv.re.v, yv.im.v);
                Cx<T> h = cxrcp(y0);
#pragma unroll
                for (int k = 0; k < K; k++) {
                    Cx<T> dp = mkcx<T>(Pre.d[k], Pim.d[k]);
                    Cx<T> dy = dp * h;
                    yv.re.d[k] = dy.re * cst<T>(-0.5);
                    yv.im.d[k] = dy.im * cst<T>(-0.5);
                }
            }
            CPair<S> YP = mkcp(yv);
            if (kind == 0) {
                S B = val(rd, rf, RF_B, RF_DB);
                S YB = yval(rd, rf, RF_YB, B);
                quartic_integrals_any<SPLIT, S, CPair<S>, WT, WX>(z, val(rd, rf, RF_LAM, RF_DLAM), val(rd, rf, RF_AA, RF_DAA),
                                                       val(rd, rf, RF_MA, RF_DMA), val(rd, rf, RF_EPSA, RF_DEPSA),
                                                       val(rd, rf, RF_RHOA, RF_DRHOA), B, P, YB, YP, qA,
                                                       val(rd, rf, RF_QB, RF_DQB), wP, nrm, Ichi, It, IX, fail);
            } else {
                cubic_integrals_any<SPLIT, S, CPair<S>, WT, WX>(z, A, P, YA, YP, amh, qA, wP, nrm, Ichi, It, IX, fail);
            }
        } else {
            wim = wim + cst<T>(1.0);
            if constexpr (K > 0) wim.v = one_plus_qz<T>(rd, rf, RF_QPIM, z);
            else wim = one_plus_qz<T>(rd, rf, RF_QPIM, z);
            RPair<S> P = mkrp<S>(Pre, Pim), wP = mkrp<S>(wre, wim);
            RPair<S> YP = mkrp<S>(yval(rd, rf, RF_YPRE, Pre), yval(rd, rf, RF_YPIM, Pim));
            if (kind == 1) {
                S B = val(rd, rf, RF_B, RF_DB);
                S YB = yval(rd, rf, RF_YB, B);
                quartic_integrals_any<SPLIT, S, RPair<S>, WT, WX>(z, val(rd, rf, RF_LAM, RF_DLAM), val(rd, rf, RF_AA, RF_DAA),
                                                       val(rd, rf, RF_MA, RF_DMA), val(rd, rf, RF_EPSA, RF_DEPSA),
                                                       val(rd, rf, RF_RHOA, RF_DRHOA), B, P, YB, YP, qA,
                                                       val(rd, rf, RF_QB, RF_DQB), wP, nrm, Ichi, It, IX, fail);
            } else {
                cubic_integrals_any<SPLIT, S, RPair<S>, WT, WX>(z, A, P, YA, YP, amh, qA, wP, nrm, Ichi, It, IX, fail);
            }
        }
    }
};


// per-pair results in the output type TO
template <class TO, int K> struct PairOut {
    TO v[N_OUT];
    TO d[N_OUT][K > 0 ? K : 1];   // tangents w.r.t. the Omega directions
    TO h0[N_OUT];                 // derivative w.r.t. H0
};

template <class TO> __device__ __forceinline__ TO load_io(const void* p, int64_t i) {
    return __ldg(reinterpret_cast<const TO*>(p) + i);
}

// Evaluate one pair.  PREC 0: FP64 throughout.  PREC 1: FP32 throughout (the
// root records come from the FP64 preparation).
template <int PREC, int K, bool WT, bool WX>
LCDM_HD void eval_pair(typename std::conditional<PREC == 0, double, float>::type zin,
                                          const double* rd, const float2* rf, PairOut<
                                          typename std::conditional<PREC == 0, double, float>::type, K>& o,
                                          int* fail) {
    typedef typename std::conditional<PREC == 0, double, float>::type TO;
    const int kind = (int)rf[RF_KIND].x;
    TO Ichi, It = 0, IX = 0;
    TO dIchi[K > 0 ? K : 1], dIt[K > 0 ? K : 1], dIX[K > 0 ? K : 1];
    {
        typedef PairEval<TO, K, WT, WX> E;
        typename E::S a, b, c;
        E::run(zin, rd, rf, kind, a, b, c, fail);
        if constexpr (K > 0) {
            Ichi = a.v; It = WT ? b.v : (TO)0; IX = WX ? c.v : (TO)0;
            for (int k = 0; k < K; k++) {
                dIchi[k] = a.d[k];
                dIt[k] = WT ? b.d[k] : (TO)0;
                dIX[k] = WX ? c.d[k] : (TO)0;
            }
        } else {
            Ichi = a; It = WT ? b : (TO)0; IX = WX ? c : (TO)0;
        }
    }
    // observables
    const TO z = zin;
    const TO H0 = recv<TO>(rd, rf, RF_H0);
    const TO DH = recv<TO>(rd, rf, RF_DH), tH = recv<TO>(rd, rf, RF_TH), Ok = recv<TO>(rd, rf, RF_OK);
    TO S, SD, Sk;
    curv_map<TO>(Ichi, Ok, S, SD, Sk);
    const TO ln10 = (TO)2.302585092994045684;
    o.v[O_DC] = DH * Ichi;
    o.v[O_T] = tH * It;
    o.v[O_X] = DH * IX;
    o.v[O_DM] = DH * S;
    o.v[O_DL] = ((TO)1 + z) * o.v[O_DM];
    o.v[O_MU] = (TO)5 * log10(o.v[O_DL]) + (TO)25;
    for (int i = 0; i < O_MU; i++) o.h0[i] = -o.v[i] / H0;
    o.h0[O_MU] = (TO)-5 / (ln10 * H0);
    if constexpr (K > 0) {
        for (int k = 0; k < K; k++) {
            TO dOk = recv<TO>(rd, rf, RF_DOK + k);
            o.d[O_DC][k] = DH * dIchi[k];
            o.d[O_T][k] = tH * dIt[k];
            o.d[O_X][k] = DH * dIX[k];
            o.d[O_DM][k] = DH * (SD * dIchi[k] + Sk * dOk);
            o.d[O_DL][k] = ((TO)1 + z) * o.d[O_DM][k];
            o.d[O_MU][k] = z == (TO)0 ? (TO)0 : (TO)5 / ln10 * o.d[O_DM][k] / o.v[O_DM];
        }
    }
}

// Warp-segmented sum of v[NV] by key (keys contiguous within the warp); the
// first lane of each segment returns true and holds the segment total.
template <int NV> __device__ __forceinline__ bool seg_reduce(double* v, int64_t key) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int64_t ok = __shfl_down_sync(full, key, off);
#pragma unroll
        for (int i = 0; i < NV; i++) {
            double o = __shfl_down_sync(full, v[i], off);
            if (lane + off < 32 && ok == key) v[i] += o;
        }
    }
    int64_t prev = __shfl_up_sync(full, key, 1);
    return lane == 0 || prev != key;
}

__device__ __forceinline__ int64_t row_search(const int64_t* __restrict__ off, int64_t B, int64_t p) {
    int64_t lo = 0, hi = B;  // off[lo] <= p < off[hi]
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= p) lo = mid; else hi = mid;
    }
    return lo;
}

// Row of an absolute pair index.
__device__ __forceinline__ int64_t row_of(const PairArgs& a, int64_t p) {
    return a.layout == LAYOUT_CSR ? row_search(a.offsets, a.B, p) : p / a.nrow;
}

// Add one row's sums v[] (ncol gradient entries, then the log-likelihood at
// index nll) from one lane: into the warp's own slot when the row is the
// warp's first or last row and the reduction is deterministic, else into the
// row's FP64 sums.
__device__ __forceinline__ void add_row(const PairArgs& a, int64_t row, const double* v, int nll, int64_t warp,
                                        int64_t wf, int64_t wl) {
    if (a.part && warp < a.det_cap && (row == wf || row == wl)) {
        double* slot = a.part + (warp * 2 + (row == wf ? 0 : 1)) * DET_SLOT;
        if (a.grad) for (int i = 0; i < a.ncol; i++) atomicAdd(slot + i, v[i]);
        if (a.loglike) atomicAdd(slot + DET_SLOT - 1, v[nll]);
        return;
    }
    if (a.grad) for (int i = 0; i < a.ncol; i++) atomicAdd(a.grad + row * a.ncol + i, v[i]);
    if (a.loglike) atomicAdd(a.loglike + row, v[nll]);
}

__device__ __forceinline__ double acc_to_double(double v) { return v; }
__device__ __forceinline__ double acc_to_double(df64 v) { return (double)v.hi + (double)v.lo; }

// Warp sum of the per-lane accumulators of one row, added to the row's FP64 sums.
// acc[i * ACC_STRIDE]: the lane's accumulators in shared memory.
enum { ACC_STRIDE = 256 };
template <int NV, int K, class AccT>
__device__ __forceinline__ void flush_row(const AccT* acc, int64_t row, const PairArgs& a, int lane, int64_t warp,
                                          int64_t wf, int64_t wl) {
    double v[NV];
#pragma unroll
    for (int i = 0; i < NV; i++) {
        v[i] = acc_to_double(acc[i * ACC_STRIDE]);
        for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], off);
    }
    if (lane == 0) add_row(a, row, v, K + 1, warp, wf, wl);
}

// Register budget: the FP32 kernels are bound by how many warps hide the
// latency of their dependent chains, so the three-tangent kernel is held to
// 128 registers (two full blocks per SM) and the value kernel to 85 (three),
// which measured faster than the unconstrained allocation (the tangent
// kernel of the benchmark step: 0.51 ms against 0.62 ms, with the pair's
// integrals inlined).
// (The kernels with X's tangents need more: they are left unconstrained.)
template <int PREC, int K, bool WX>
struct MinBlocks { enum { value = PREC == 1 ? ((K == 3 && !WX) ? 2 : (K == 0 ? 3 : 1)) : 1 }; };

template <int PREC, int K, bool WT, bool WX>
__global__ void __launch_bounds__(256, MinBlocks<PREC, K, WX>::value) pairs_kernel(PairArgs a) {
    typedef typename std::conditional<PREC == 0, double, float>::type TO;
    constexpr int NV = K + 2;   // H0, K Omega directions, loglike value
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t start = warp * a.chunk;
    const int64_t end = max(start, min(start + a.chunk, a.nnz));   // empty range past the end
    const bool reduce = (a.grad != nullptr) || (a.loglike != nullptr);
    const bool loglike = a.mobs != nullptr;
    const TO inv_sig = (TO)(1.0 / a.sigma);
    const TO lnorm = (TO)(-log(a.sigma * 2.5066282746310002));
    const TO Mobs = (TO)a.M;
    typedef typename std::conditional<PREC == 0, double, df64>::type AccT;
    int64_t row = -1;
    // The per-lane accumulators live in shared memory (lane-private slots):
    // they would otherwise stay in registers through the whole pair
    // evaluation, where registers bound the number of resident warps.
    __shared__ AccT acc_s[NV * ACC_STRIDE];
    AccT* acc = acc_s + threadIdx.x;
    int64_t acc_row = -1;
#pragma unroll
    for (int i = 0; i < NV; i++) acc[i * ACC_STRIDE] = cst<AccT>(0.0);
    // deterministic reduction: the warp's first and last rows, its slots zeroed
    int64_t wf = -1, wl = -1;
    if (a.part && reduce && warp < a.det_cap) {
        if (start < end) {
            wf = row_of(a, a.base + start);
            wl = row_of(a, a.base + end - 1);
        }
        if (lane < 2 * DET_SLOT) a.part[warp * 2 * DET_SLOT + lane] = 0.0;
        if (lane < 2) a.wrow[warp * 2 + lane] = lane == 0 ? wf : wl;
        __syncwarp();
        __threadfence_block();
    }
    const int64_t len = end - start, nb = (len + 31) / 32, nb_all = a.chunk / 32;
    const int64_t s_lane = a.interleave ? nb : 1, s_it = a.interleave ? 1 : 32;
    // With a full-SM block (256 threads) the warps of the kernels whose code per
    // pair is largest (X's tangents, seven-column tangents) step through their
    // ranges together, one 32-pair batch at a time: that code is about the size
    // of the instruction cache, and warps at the same place in it share each
    // fetched line.  Every warp then runs nb_all steps (the same number).  For
    // the other kernels the barrier costs more than it saves (measured).
    const bool lockstep = blockDim.x == 256 && K > 0 && (WX || K > 3);
    for (int64_t it = 0; it < nb_all; it++) {
        if (lockstep) __syncthreads();
        if (it >= nb) continue;
        const int64_t off = (int64_t)lane * s_lane + it * s_it;
        const bool active = off < len;
        const int64_t lidx = start + (active ? off : len - 1);
        const int64_t pidx = a.base + lidx;                  // absolute pair index
        const int64_t pp = pidx;
        int64_t zi = pp;
        if (a.layout == LAYOUT_CSR) {
            if (row < 0) {
                row = row_search(a.offsets, a.B, pp);
            } else {
                int steps = 0;
                while (row < a.B - 1 && __ldg(a.offsets + row + 1) <= pp && steps < 8) { row++; steps++; }
                if (row < a.B - 1 && __ldg(a.offsets + row + 1) <= pp) row = row_search(a.offsets, a.B, pp);
            }
        } else {
            row = pp / a.nrow;
            if (a.layout == LAYOUT_SHARED) zi = pp - row * a.nrow;
        }
        const double* rd = a.recD + row * NREC;
        const float2* rf = a.recF + row * NREC;
        const int st = a.status[row];
        const TO z = load_io<TO>(a.z, zi);
        // the pair's cotangents (or observed magnitude) are loaded before the
        // evaluation, so that their latency hides behind it
        TO gcot[N_OUT];
        TO mob = (TO)0;
        if constexpr (K > 0) {
#pragma unroll
            for (int i = 0; i < N_OUT; i++) gcot[i] = (reduce && !loglike && a.cot[i]) ? load_io<TO>(a.cot[i], pidx) : (TO)0;
            if (loglike) mob = load_io<TO>(a.mobs, zi);
        }
        PairOut<TO, K> o;
        int fail = 0;
        if (st == ST_OK) {
            if (z == (TO)0) {
                for (int i = 0; i < N_OUT; i++) { o.v[i] = 0; o.h0[i] = 0; for (int k = 0; k < (K > 0 ? K : 1); k++) o.d[i][k] = 0; }
                o.v[O_MU] = -CUDART_INF;
                o.h0[O_MU] = (TO)(-5.0 / (2.302585092994045684 * rd[RF_H0]));
            } else {
                eval_pair<PREC, K, WT, WX>(z, rd, rf, o, &fail);
            }
        }
        if (st != ST_OK || fail) {
            const TO nan = (TO)CUDART_NAN;
            for (int i = 0; i < N_OUT; i++) { o.v[i] = nan; o.h0[i] = nan; for (int k = 0; k < (K > 0 ? K : 1); k++) o.d[i][k] = nan; }
            if (fail && active && st == ST_OK) atomicMax(a.status + row, (int)ST_NOCONV);
        }
        if (active) {
#pragma unroll
            for (int i = 0; i < N_OUT; i++) {
                if (a.outmask & (1 << i)) reinterpret_cast<TO*>(a.out[i])[pidx] = o.v[i];
                if (K > 0 && a.jac[i]) {
                    TO* jp = reinterpret_cast<TO*>(a.jac[i]) + pidx * a.ncol;
                    jp[0] = o.h0[i];
                    for (int k = 0; k < K; k++) jp[1 + k] = o.d[i][k];
                }
            }
        }
        if (!reduce) continue;
        // contribution of this pair to the per-cosmology sums
        TO c[NV];
#pragma unroll
        for (int i = 0; i < NV; i++) c[i] = 0;
        if (active && st == ST_OK && !fail) {
            if (loglike) {
                TO r = ((K > 0 ? mob : load_io<TO>(a.mobs, zi)) - o.v[O_MU] - Mobs) * inv_sig;
                TO w = r * inv_sig;
                c[0] = w * o.h0[O_MU];
#pragma unroll
                for (int k = 0; k < K; k++) c[1 + k] = w * o.d[O_MU][k];
                c[K + 1] = (TO)-0.5 * r * r + lnorm;
            } else {
#pragma unroll
                for (int i = 0; i < N_OUT; i++) {
                    if (!a.cot[i]) continue;
                    TO g = K > 0 ? gcot[i] : load_io<TO>(a.cot[i], pidx);
                    c[0] += g * o.h0[i];
#pragma unroll
                    for (int k = 0; k < K; k++) c[1 + k] += g * o.d[i][k];
                }
            }
        }
        // register accumulation while the whole warp stays on one row
        const int64_t r0 = __shfl_sync(0xffffffffu, row, 0);
        const bool uniform = __all_sync(0xffffffffu, row == r0);
        if (uniform && r0 == acc_row) {
#pragma unroll
            for (int i = 0; i < NV; i++) acc[i * ACC_STRIDE] = acc[i * ACC_STRIDE] + c[i];
            continue;
        }
        if (acc_row >= 0) flush_row<NV, K>(acc, acc_row, a, lane, warp, wf, wl);
        if (uniform) {
#pragma unroll
            for (int i = 0; i < NV; i++) acc[i * ACC_STRIDE] = cst<AccT>(0.0) + c[i];
            acc_row = r0;
        } else {
            double cd_[NV];
#pragma unroll
            for (int i = 0; i < NV; i++) cd_[i] = (double)c[i];
            if (seg_reduce<NV>(cd_, row) && active) add_row(a, row, cd_, K + 1, warp, wf, wl);
#pragma unroll
            for (int i = 0; i < NV; i++) acc[i * ACC_STRIDE] = cst<AccT>(0.0);
            acc_row = -1;
        }
    }
    if (reduce && acc_row >= 0) flush_row<NV, K>(acc, acc_row, a, lane, warp, wf, wl);
}

}  // namespace lcdm
