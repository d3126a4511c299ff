// General integration limits (eqs. 2.3-2.5 from z1 to z2) and the upper
// limit at infinity, on top of the z1 = 0 path.
//
// For a lower limit z1 the substitution 1+z = (1+z1)(1+z') maps the integrals
// over [z1, z2] onto integrals over [0, z'] of a closed cosmology: with
// s = 1+z1 and E1 = E^2(z1),
//   Omega'_m = Omega_m s^3 / E1, Omega'_L = Omega_L / E1, Omega'_r = Omega_r s^4 / E1,
//   Omega'_k = Omega_k s^2 / E1, H0' = H0 sqrt(E1), z' = (z2 - z1) / s,
// the roots move to r' = (r - z1) / s, and
//   chi(z1, z2) = s chi'(0, z'),  t(z1, z2) = t'(0, z'),  d_abs(z1, z2) = s^3 d_abs'(0, z'),
//   d_M(z1, z2) = s d_M'(z'),  and d_L'(z') = (1+z2) d_M(z1, z2) / (1+z1)^2 is the
//   luminosity distance of a source at z2 seen by a comoving observer at z1.
// Substituted into the definitions of Sec. 3.1 this is eqs. (3.7)-(3.9) with
// X_m = sqrt(z2 - r_m), Y_m = sqrt(z1 - r_m), every factor of s cancelling:
// the same formulas, evaluated in the observer's own coordinate.  So the
// per-pair kernels run unchanged on the shifted cosmology (one row each) and
// small kernels here do the per-row shift, the per-pair map of z and of the
// cotangents, the output scaling, and the chain rule of the gradient.
//
// The shifted Omega' sum to one identically (E^2(z1) / E1), so the shifted
// row takes the closure form (H0', Om', OL', Or') with Ok' = 1 - Om' - OL' -
// Or', and the same three-direction tangents as a closure row: because
// sum_i dOmega'_i / dtheta = 0, the chain rule needs only the closure
// derivatives d/dOmega'_a - d/dOk' (a = m, L, r).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lcdm {

struct ShiftArgs {
    const double* params;   // [B][ncol]
    const double* z1;       // [B]
    int64_t B;
    int ncol;
    double* params4;        // [B][4] (H0', Om', OL', Or'), closure
    double* jac;            // [B][4][ncol] d params4 / d params
    double* scale;          // [B] s = 1 + z1 (NaN for an invalid row)
    float4* rowf;           // [B] (z1 hi, z1 lo, 1/s, s) in float32 for the FP32 pair maps
};

struct PairMapArgs {
    const int64_t* offsets; // CSR offsets, or null for the dense layout
    int64_t nrow;           // pairs per row (dense)
    int64_t nnz;
    int64_t B;
    int fp64;               // z, outputs and cotangents are float64 (else float32)
    const double* z1;       // [B]
    const double* scale;    // [B]
    const float4* rowf;     // [B] float32 row constants (FP32 maps)
    const void* z2;         // [nnz]
    void* zp;               // [nnz] z' = (z2 - z1) / s
    const void* cot[6];     // user cotangents
    void* cotp[6];          // scaled cotangents (d_C, X, d_M; null = not needed)
    void* out[6];           // outputs scaled in place
};

struct LimitArgs {
    const double* recD;     // records of the shifted cosmologies
    const float2* recF;
    int32_t* status;
    int64_t B;
    const double* scale;
    double* chi;            // [B] chi(z1, inf), Mpc (may be null)
    double* age;            // [B] t(z1, inf), Gyr (may be null)
    const double* cot_chi;  // [B] (VJP; may be null)
    const double* cot_age;
    double* gradp;          // [B][4] gradient w.r.t. the shifted parameters (VJP)
};

cudaError_t launch_shift(const ShiftArgs& a, cudaStream_t s);
cudaError_t launch_pair_pre(const PairMapArgs& a, cudaStream_t s);
cudaError_t launch_pair_post(const PairMapArgs& a, cudaStream_t s);
cudaError_t launch_chain(const double* jac, const double* gradp, int64_t B, int ncol, double* grad,
                         cudaStream_t s);
cudaError_t launch_limits(const LimitArgs& a, bool tangents, cudaStream_t s);

}  // namespace lcdm
