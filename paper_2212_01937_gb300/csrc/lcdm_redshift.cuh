// Derivatives with respect to the redshift of a pair (the upper limit z2 of
// eqs. 2.3-2.5), for models whose redshifts are themselves parameters (the
// latent redshifts of the Sec. 4 supernova model).  By the fundamental
// theorem of calculus the derivative of an integral with respect to its
// upper limit is the integrand there: d chi / dz = (c/H0) / E(z).  Through
// the curvature map and the luminosity distance:
//   d mu / dz = (5 / ln 10) [ 1/(1+z) + S_k'(D) / (E(z) S_k(D)) ],
// D = chi H0 / c, S_k as in the observables (d_M = (c/H0) S_k(D)).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lcdm {

struct DzArgs {
    const double* params;   // [B][ncol]
    int ncol;
    const int32_t* status;  // [B]
    const int64_t* offsets; // CSR offsets, or null (dense / shared: nrow pairs per row)
    int layout;             // Layout of the pair kernel
    int64_t nrow, nnz, B;
    int fp64;
    const void* z;          // [n] (shared) or [nnz]
    const void* mobs;       // like z
    const void* dC;         // [nnz] comoving distance of each pair
    const void* mu;         // [nnz] distance modulus of each pair (likelihood mode)
    double M, sigma;
    const void* cot[6];     // VJP mode: cotangents of the six outputs (null = zero)
    int vjp;                // 0: likelihood mode, 1: VJP mode
    void* grad_z;           // [nnz] d loglike_row / d z_pair, or sum_o cot_o d out_o / dz
};

// Likelihood mode: grad_z = (m_obs - mu - M) / sigma^2 * d mu/dz.
// VJP mode: grad_z = sum_o cot_o d out_o/dz with
//   d chi/dz = (c/H0)/E, d t/dz = 1/(H0 (1+z) E), d d_abs/dz = (c/H0)(1+z)^2/E,
//   d d_M/dz = (c/H0) S_k'(D)/E, d d_L/dz = d_M + (1+z) d d_M/dz, d mu/dz as above
//   (0 at z = 0, where mu = -inf).
cudaError_t launch_loglike_dz(const DzArgs& a, cudaStream_t s);

}  // namespace lcdm
