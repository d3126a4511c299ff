// Per-pair derivatives with respect to the pair's redshift: of the Gaussian
// log-likelihood of magnitudes (Sec. 4), or of a cotangent-weighted sum of
// the outputs; see lcdm_redshift.cuh.
#include <math_constants.h>

#include "lcdm_kernels.cuh"
#include "lcdm_redshift.cuh"

namespace lcdm {

template <class T> __global__ void __launch_bounds__(256) loglike_dz_kernel(DzArgs a) {
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    int64_t chunk = (a.nnz + nw - 1) / nw;
    chunk = (chunk + 31) / 32 * 32;
    const int64_t p0 = min(a.nnz, w * chunk), p1 = min(a.nnz, p0 + chunk);
    const T ln10 = (T)2.302585092994045684, c5 = (T)5 / ln10, inv_s2 = (T)(1.0 / (a.sigma * a.sigma));
    int64_t row = -1;
    for (int64_t p = p0 + (threadIdx.x & 31); p < p1; p += 32) {
        // row of pair p: binary search once, then step forward
        if (a.layout == LAYOUT_CSR) {
            if (row < 0) {
                int64_t lo = 0, hi = a.B;
                while (hi - lo > 1) {
                    int64_t mid = (lo + hi) >> 1;
                    if (__ldg(a.offsets + mid) <= p) lo = mid; else hi = mid;
                }
                row = lo;
            }
            while (row < a.B - 1 && __ldg(a.offsets + row + 1) <= p) row++;
        } else {
            if (row < 0) row = p / a.nrow;
            while ((row + 1) * a.nrow <= p) row++;
        }
        const int64_t zi = a.layout == LAYOUT_SHARED ? p - row * a.nrow : p;
        T* out = reinterpret_cast<T*>(a.grad_z) + p;
        if (a.status[row] != ST_OK) { *out = (T)CUDART_NAN; continue; }
        const double* pr = a.params + row * a.ncol;
        const T Om = (T)pr[1], OL = (T)pr[2], Or = (T)pr[3];
        const T Ok = a.ncol == 5 ? (T)pr[4] : (T)(1.0 - pr[1] - pr[2] - pr[3]);
        const T z = reinterpret_cast<const T*>(a.z)[zi];
        if (z == (T)0 && !a.vjp) { *out = (T)0; continue; }   // mu = -inf there: no finite derivative
        const T x = (T)1 + z, x2 = x * x;
        const T E = sqrt(((Or * x + Om) * x + Ok) * x2 + OL);          // eq. (2.2)
        const T DH = (T)(LCDM_C_KMS / pr[0]);
        const T D = reinterpret_cast<const T*>(a.dC)[p] / DH;
        T S, SD, Sk;
        curv_map<T>(D, Ok, S, SD, Sk);
        const T dmu = z == (T)0 ? (T)0 : c5 * ((T)1 / x + SD / (E * S));
        if (!a.vjp) {
            const T mu = reinterpret_cast<const T*>(a.mu)[p];
            const T r = reinterpret_cast<const T*>(a.mobs)[zi] - mu - (T)a.M;
            *out = r * inv_s2 * dmu;
            continue;
        }
        // the integrands of eqs. (2.3)-(2.5) at the upper limit, then the observables
        const T iE = (T)1 / E;
        const T dM = DH * SD * iE;
        const T d[6] = {DH * iE, (T)(LCDM_HUBBLE_GYR / pr[0]) * iE / x, DH * x2 * iE, dM, DH * S + x * dM, dmu};
        T g = 0;
#pragma unroll
        for (int o = 0; o < 6; o++)
            if (a.cot[o]) g += reinterpret_cast<const T*>(a.cot[o])[p] * d[o];
        *out = g;
    }
}

cudaError_t launch_loglike_dz(const DzArgs& a, cudaStream_t s) {
    if (a.nnz <= 0) return cudaSuccess;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t need = (a.nnz + 255) / 256, cap = (int64_t)sms * 8;
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    if (a.fp64) loglike_dz_kernel<double><<<grid, 256, 0, s>>>(a);
    else loglike_dz_kernel<float><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lcdm
