// Kernels of the general-limits path (see lcdm_between.cuh): the per-row
// shift of the parameters, the per-pair maps, the gradient chain rule, and
// the upper limit at infinity (age and horizon, FP64, one thread per row).
#include <math_constants.h>

#include "lcdm_between.cuh"
#include "lcdm_kernels.cuh"

namespace lcdm {

// ------------------------------------------------------------ row shift ----
__global__ void shift_kernel(ShiftArgs a) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.B) return;
    const int nc = a.ncol;
    const double* p = a.params + b * nc;
    const double H0 = p[0], Om = p[1], OL = p[2], Or = p[3];
    const double Ok = nc == 5 ? p[4] : 1.0 - Om - OL - Or;
    const double z1 = a.z1[b];
    const double s = 1.0 + z1, s2 = s * s, s3 = s2 * s, s4 = s2 * s2;
    // E^2(z1), eq. (2.2); exactly 1 at z1 = 0 under the closure
    const double E1 = (z1 == 0.0 && nc == 4) ? 1.0 : Or * s4 + Om * s3 + Ok * s2 + OL;
    double* q = a.params4 + b * 4;
    double* J = a.jac + b * 4 * nc;
    if (!(z1 >= 0.0) || !isfinite(z1) || !(E1 > 0.0) || !isfinite(E1)) {
        const double nan = CUDART_NAN;
        for (int i = 0; i < 4; i++) q[i] = nan;
        for (int i = 0; i < 4 * nc; i++) J[i] = nan;
        a.scale[b] = nan;
        a.rowf[b] = make_float4(nan, nan, nan, nan);
        return;
    }
    const double iE = 1.0 / E1, rE = sqrt(E1);
    const double pw[4] = {s3, 1.0, s4, s2};       // powers of s for (Om, OL, Or, Ok)
    const double om[4] = {Om, OL, Or, Ok};
    q[0] = H0 * rE;
    for (int i = 0; i < 3; i++) q[1 + i] = om[i] * pw[i] * iE;
    // derivatives: column 0 is H0; the Omega columns act on (Om, OL, Or[, Ok]),
    // with dOk = -1 for each of the first three under the closure
    J[0 * nc + 0] = rE;
    for (int i = 0; i < 3; i++) J[(1 + i) * nc + 0] = 0.0;
    for (int c = 1; c < nc; c++) {
        double d[4] = {0.0, 0.0, 0.0, 0.0};
        d[c - 1] = 1.0;
        if (nc == 4) d[3] = -1.0;
        double dE = 0.0;
        for (int i = 0; i < 4; i++) dE += pw[i] * d[i];
        J[0 * nc + c] = 0.5 * H0 * dE / rE;
        for (int i = 0; i < 3; i++) J[(1 + i) * nc + c] = (pw[i] * d[i] - q[1 + i] * dE) * iE;
    }
    a.scale[b] = s;
    // z1 as an unevaluated float sum hi + lo, so that z2 - z1 and the sign test
    // z2 >= z1 come out right in float32 arithmetic when z2 is close to z1
    const float hi = (float)z1;
    a.rowf[b] = make_float4(hi, (float)(z1 - (double)hi), (float)(1.0 / s), (float)s);
}

cudaError_t launch_shift(const ShiftArgs& a, cudaStream_t s) {
    if (a.B <= 0) return cudaSuccess;
    shift_kernel<<<(unsigned)((a.B + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------- per-pair maps -----
// Each warp takes a contiguous run of pairs, lane l every 32nd pair from l
// (coalesced); the row of a lane's first pair comes from a binary search of
// the CSR offsets, later rows from stepping forward.
struct RowWalk {
    const int64_t* off;
    int64_t B, nrow, row;
    __device__ int64_t at(int64_t p) {
        if (!off) {
            if (row < 0) row = p / nrow;
            while ((row + 1) * nrow <= p) row++;
            return row;
        }
        if (row < 0) {
            int64_t lo = 0, hi = B;   // off[lo] <= p < off[hi]
            while (hi - lo > 1) {
                int64_t mid = (lo + hi) >> 1;
                if (__ldg(off + mid) <= p) lo = mid; else hi = mid;
            }
            row = lo;
        }
        while (row < B - 1 && __ldg(off + row + 1) <= p) row++;
        return row;
    }
};

#define LCDM_MAP_BLOCK 256
#define LCDM_MAP_BLOCKS_PER_SM 8

__device__ __forceinline__ void warp_run(int64_t nnz, int64_t& p0, int64_t& p1) {
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    int64_t chunk = (nnz + nw - 1) / nw;
    chunk = (chunk + 31) / 32 * 32;
    p0 = min(nnz, w * chunk);
    p1 = min(nnz, p0 + chunk);
}

// z' = (z2 - z1) / s, the domain test z2 >= z1, and the output / cotangent
// factors (s for d_C and d_M, s^3 for d_abs, 1 otherwise), in the pass type
template <class T> struct RowMap;
template <> struct RowMap<float> {
    float hi, lo, is, s;
    __device__ RowMap(const PairMapArgs& a, int64_t b) {
        const float4 r = a.rowf[b];
        hi = r.x; lo = r.y; is = r.z; s = r.w;
    }
    // (z2 - hi) is exact near z1 (Sterbenz) and its sign is exact; lo is
    // |z1 - hi| rounded, which keeps the sign of the tie z2 == hi
    __device__ float dz(float z2) const { return (z2 - hi) - lo; }
    __device__ float zp(float d) const { return d * is; }
    __device__ float f(int o) const { return o == 2 ? s * s * s : ((o == 0 || o == 3) ? s : 1.0f); }
};
template <> struct RowMap<double> {
    double z1, s;
    __device__ RowMap(const PairMapArgs& a, int64_t b) : z1(a.z1[b]), s(a.scale[b]) {}
    __device__ double dz(double z2) const { return z2 - z1; }
    __device__ double zp(double d) const { return d / s; }
    __device__ double f(int o) const { return o == 2 ? s * s * s : ((o == 0 || o == 3) ? s : 1.0); }
};

template <class T> __global__ void __launch_bounds__(LCDM_MAP_BLOCK) pair_pre_kernel(PairMapArgs a) {
    int64_t p0, p1;
    warp_run(a.nnz, p0, p1);
    RowWalk rw{a.offsets, a.B, a.nrow, -1};
    for (int64_t p = p0 + (threadIdx.x & 31); p < p1; p += 32) {
        const RowMap<T> m(a, rw.at(p));
        const T d = m.dz(reinterpret_cast<const T*>(a.z2)[p]);
        // an interval with z2 < z1 is outside the domain: evaluated at z' = 0,
        // its outputs are set to NaN afterwards and it adds nothing to the gradient
        const bool ok = d >= (T)0;
        reinterpret_cast<T*>(a.zp)[p] = ok ? m.zp(d) : (T)0;
#pragma unroll
        for (int o = 0; o < 6; o++)
            if (a.cotp[o]) {
                const T g = reinterpret_cast<const T*>(a.cot[o])[p];
                reinterpret_cast<T*>(a.cotp[o])[p] = ok ? m.f(o) * g : (T)0;
            }
    }
}

template <class T> __global__ void __launch_bounds__(LCDM_MAP_BLOCK) pair_post_kernel(PairMapArgs a) {
    int64_t p0, p1;
    warp_run(a.nnz, p0, p1);
    RowWalk rw{a.offsets, a.B, a.nrow, -1};
    for (int64_t p = p0 + (threadIdx.x & 31); p < p1; p += 32) {
        const RowMap<T> m(a, rw.at(p));
        const bool ok = m.dz(reinterpret_cast<const T*>(a.z2)[p]) >= (T)0;
        // t, d_L and mu need no factor: they are touched only to mark a pair
        // outside the domain
#pragma unroll
        for (int o = 0; o < 6; o++)
            if (a.out[o]) {
                T* v = reinterpret_cast<T*>(a.out[o]) + p;
                if (!ok) *v = (T)CUDART_NAN;
                else if (o == 0 || o == 2 || o == 3) *v = m.f(o) * *v;
            }
    }
}

static unsigned map_grid(int64_t nnz) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t need = (nnz + LCDM_MAP_BLOCK - 1) / LCDM_MAP_BLOCK, cap = (int64_t)sms * LCDM_MAP_BLOCKS_PER_SM;
    return (unsigned)(need < cap ? (need > 0 ? need : 1) : cap);
}

cudaError_t launch_pair_pre(const PairMapArgs& a, cudaStream_t s) {
    if (a.nnz <= 0) return cudaSuccess;
    if (a.fp64) pair_pre_kernel<double><<<map_grid(a.nnz), LCDM_MAP_BLOCK, 0, s>>>(a);
    else pair_pre_kernel<float><<<map_grid(a.nnz), LCDM_MAP_BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pair_post(const PairMapArgs& a, cudaStream_t s) {
    if (a.nnz <= 0) return cudaSuccess;
    if (a.fp64) pair_post_kernel<double><<<map_grid(a.nnz), LCDM_MAP_BLOCK, 0, s>>>(a);
    else pair_post_kernel<float><<<map_grid(a.nnz), LCDM_MAP_BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------ gradient chain -----
// grad[b][c] = sum_a gradp[b][a] d params4[b][a] / d params[b][c].  Entries
// with a zero Jacobian are skipped, so that the NaN Omega_r' component of a
// radiationless row (no such direction in the cubic) reaches only the
// Omega_r column, as on the z1 = 0 path.
__global__ void chain_kernel(const double* __restrict__ jac, const double* __restrict__ gradp, int64_t B,
                             int ncol, double* __restrict__ grad) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double* J = jac + b * 4 * ncol;
    const double* g = gradp + b * 4;
    for (int c = 0; c < ncol; c++) {
        double acc = 0.0;
        for (int i = 0; i < 4; i++) {
            const double j = J[i * ncol + c];
            if (j != 0.0) acc += g[i] * j;
        }
        grad[b * ncol + c] = acc;
    }
}

cudaError_t launch_chain(const double* jac, const double* gradp, int64_t B, int ncol, double* grad,
                         cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    chain_kernel<<<(unsigned)((B + 127) / 128), 128, 0, s>>>(jac, gradp, B, ncol, grad);
    return cudaGetLastError();
}

// ------------------------------------------------- upper limit at infinity -
// One thread per row of the shifted cosmology: chi'(0, inf) and t'(0, inf)
// in FP64, with the closure tangents w.r.t. (Om', OL', Or') when K = 3.
template <int K> struct LimitEval {
    typedef PairEval<double, K, true, false> E;
    typedef typename E::S S;

    static __device__ void run(const double* rd, const float2* rf, int kind, S& Ichi, S& It, int* fail) {
        S A = E::val(rd, rf, RF_A, RF_DA);
        S amh = E::val(rd, rf, RF_AMH, RF_DAMH);
        S Pre = E::val(rd, rf, RF_PRE, RF_DPRE), Pim = E::val(rd, rf, RF_PIM, RF_DPIM);
        S qA = E::val(rd, rf, RF_QA, RF_DQA), nrm = E::val(rd, rf, RF_NRM, RF_DNRM);
        S qPre = E::val(rd, rf, RF_QPRE, RF_DQPRE), qPim = E::val(rd, rf, RF_QPIM, RF_DQPIM);
        if (kind == 0 || kind == 2) {
            CPair<S> P = mkcp(mkcx<S>(Pre, Pim)), qP = mkcp(mkcx<S>(qPre, qPim));
            if (kind == 0)
                quartic_limits<S, CPair<S> >(E::val(rd, rf, RF_MA, RF_DMA), E::val(rd, rf, RF_EPSA, RF_DEPSA),
                                             E::val(rd, rf, RF_B, RF_DB), P, qA, E::val(rd, rf, RF_QB, RF_DQB),
                                             qP, nrm, Ichi, It, fail);
            else
                cubic_limits<S, CPair<S> >(A, amh, qA, qP, nrm, Ichi, It, fail);
        } else {
            RPair<S> P = mkrp<S>(Pre, Pim), qP = mkrp<S>(qPre, qPim);
            if (kind == 1)
                quartic_limits<S, RPair<S> >(E::val(rd, rf, RF_MA, RF_DMA), E::val(rd, rf, RF_EPSA, RF_DEPSA),
                                             E::val(rd, rf, RF_B, RF_DB), P, qA, E::val(rd, rf, RF_QB, RF_DQB),
                                             qP, nrm, Ichi, It, fail);
            else
                cubic_limits<S, RPair<S> >(A, amh, qA, qP, nrm, Ichi, It, fail);
        }
    }
};

template <int K> __global__ void __launch_bounds__(128) limits_kernel(LimitArgs a) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.B) return;
    const double* rd = a.recD + b * NREC;
    const float2* rf = a.recF + b * NREC;
    const double nan = CUDART_NAN;
    double chi = nan, age = nan;
    int st = a.status[b];
    if (st == ST_OK) {
        typedef typename LimitEval<K>::S S;
        S Ichi, It;
        int fail = 0;
        LimitEval<K>::run(rd, rf, (int)rd[RF_KIND], Ichi, It, &fail);
        const double s = a.scale[b], DH = rd[RF_DH], tH = rd[RF_TH], H0 = rd[RF_H0];
        if (fail) {
            a.status[b] = st = ST_NOCONV;
        } else if constexpr (K > 0) {
            chi = s * DH * Ichi.v;
            age = tH * It.v;
            const double gc = a.cot_chi ? a.cot_chi[b] : 0.0, ga = a.cot_age ? a.cot_age[b] : 0.0;
            double* g = a.gradp + b * 4;
            g[0] = -(gc * chi + ga * age) / H0;
            for (int k = 0; k < K; k++) g[1 + k] = gc * s * DH * Ichi.d[k] + ga * tH * It.d[k];
        } else {
            chi = s * DH * Ichi;
            age = tH * It;
        }
    }
    if (st != ST_OK && K > 0 && a.gradp)
        for (int k = 0; k < 4; k++) a.gradp[b * 4 + k] = nan;
    if (a.chi) a.chi[b] = chi;
    if (a.age) a.age[b] = age;
}

cudaError_t launch_limits(const LimitArgs& a, bool tangents, cudaStream_t s) {
    if (a.B <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((a.B + 127) / 128);
    if (tangents) limits_kernel<3><<<grid, 128, 0, s>>>(a);
    else limits_kernel<0><<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lcdm
