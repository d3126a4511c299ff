/*
 * lcdm.h -- C ABI of liblcdm: LambdaCDM+radiation+curvature distances for many
 * (cosmology, redshift) pairs on one GB300 (sm_103a), after Karchev,
 * "Analytic auto-differentiable LambdaCDM cosmography" (arXiv:2212.01937).
 *
 * What is computed (z1 = 0, z2 = z for every pair; lcdm_distances_between
 * and lcdm_limits below take general lower limits and z2 = infinity):
 *   comoving distance  d_C = chi(0, z)                eq. (2.3), via eq. (3.7)/(B.1)
 *   time coordinate    t   = t(0, z) (lookback time)  eq. (2.4), via eq. (3.8)/(B.2)
 *   absorption dist.   X   = d_abs(0, z)              eq. (2.5), via eq. (3.9)/(B.3)
 *   transverse comoving distance d_M (curvature map), luminosity distance
 *   d_L = (1+z) d_M and distance modulus mu = 5 log10(d_L / 10 pc)
 *                                                       (Sec. 2.1.1; fn22)
 * The quartic E^2 of eq. (2.2) is factorised per cosmology (eq. 3.2, FP64) and
 * each integral is reduced to Carlson's R_F, R_J, R_D, R_C (eqs. 2.6-2.9),
 * evaluated by duplication.  Derivatives with respect to the parameters are
 * carried through the duplication sequences as forward-mode tangents (the
 * differentiated form of eqs. 2.6-2.9; eq. 2.10 for R_C) from the root
 * derivatives of App. A (eqs. A.1-A.4).
 *
 * Conventions shared by every entry point
 *   params   [B][ncol] float64, row-major: (H0 [km/s/Mpc], Omega_m0,
 *            Omega_L0, Omega_r0) with Omega_k0 = 1 - Om - OL - Or (closure,
 *            Sec. 2.1) when ncol == 4, or a fifth column Omega_k0 (ncol == 5).
 *            Omega_r0 == 0 selects the cubic formulas of App. B.1.
 *            ncol == 7 adds, after an explicit Omega_k0, the two further
 *            components that keep E^2 a quartic (fn4): Omega_s0 (w = -1/3,
 *            scaling as (1+z)^2 like curvature but outside the curvature map)
 *            and Omega_x0 (w = -2/3, scaling as (1+z)); every density is then
 *            explicit and an independent direction of the gradients
 *            (Jacobian columns H0, Om, OL, Or, Ok, Os, Ox).  The general
 *            limits (lcdm_distances_between, lcdm_limits) and the redshift
 *            derivatives (lcdm_gauss_loglike_dz, lcdm_distances_vjp_dz) take
 *            four or five columns and return LCDM_ERR_UNSUPPORTED for seven.
 *   pairs    layout LCDM_LAYOUT_CSR: offsets[B+1] int64 (offsets[0] = 0,
 *            non-decreasing, offsets[B] = n), z[n]; row b holds pairs
 *            offsets[b] .. offsets[b+1]-1.  Empty rows are allowed.
 *            LCDM_LAYOUT_DENSE: offsets ignored, every row holds n redshifts,
 *            z[B*n].  LCDM_LAYOUT_SHARED: offsets ignored, all rows share the
 *            n redshifts z[n]; pair (b, i) has index b*n + i.
 *            npairs = n (CSR) or B*n (DENSE, SHARED).
 *   dtype    precision LCDM_FP64: z, outputs, cotangents, Jacobians and
 *            m_obs are float64 and every step is FP64.  LCDM_FP32_MIXED: they
 *            are float32 and the per-pair arithmetic is FP32 (division and
 *            square root within 2 ulp, subnormal results flushed to zero);
 *            the root solve and all per-cosmology reductions stay FP64.
 *   domain   z >= 0 (the integrals run from 0 to z); outputs for negative z
 *            are unspecified.
 *   units    d_C, d_M, d_L, X in Mpc; t in Gyr; mu in magnitudes.
 *   memory   every pointer argument except opts is a DEVICE pointer owned by
 *            the caller; the library allocates nothing.  Scratch comes from
 *            the caller's workspace ws (>= lcdm_workspace_size bytes,
 *            256-byte aligned) and must not be used concurrently by two calls.
 *   streams  calls enqueue kernels on `stream` and return without
 *            synchronising; results are ready when the stream reaches them.
 *   errors   the return value reports argument and launch errors only
 *            (LCDM_OK ... LCDM_ERR_UNSUPPORTED, see lcdm_status_string);
 *            nothing is enqueued when an argument check fails.  Per-cosmology
 *            problems are reported in cosmo_status[B] (int32, device):
 *              0 ok
 *              1 no Big Bang: a real root of E^2 at z >= 0 (Sec. 3, Fig. 1)
 *              2 invalid parameters (non-finite, H0 <= 0, Omega_r0 < 0, or
 *                Omega_m0 <= 0 when Omega_r0 == 0)
 *              3 degenerate roots (two roots coinciding exactly, other
 *                than the cases below, or rho_A == 0)
 *              4 duplication did not converge / principal value not available
 *              5 root configuration not supported (two complex pairs)
 *            and every output of such a cosmology is NaN.
 *   triple root  Omega_L0 = Omega_k0 (+ Omega_s0) = Omega_x0 = 0 to within
 *            the rounding of the closure (Einstein-de Sitter, flat matter +
 *            radiation: E^2 = x^3 (Or x + Om), x = 1 + z): the roots are set
 *            exactly and the values are computed as for any row (status 0);
 *            the root derivatives of App. A are singular there, so the
 *            gradient entries of such a row in the density directions are
 *            NaN (the H0 entry is finite).
 *   Omega_L0 = 0 with Omega_k0 != 0 (a double root at x = 0): values and
 *            FP64 gradients as for any row; in FP32 the d / d Omega_L0 entry
 *            is NaN (the root derivatives there exceed the FP32 range).
 *   z = 0    gives d = t = X = 0, mu = -inf; tangents of mu with respect to
 *            the Omega columns are 0 and d mu / d H0 = -5 / (H0 ln 10).
 *   gradient with respect to Omega_r0 of a radiationless cosmology
 *            (Omega_r0 == 0) is NaN: the cubic reduction has no such direction.
 */
#ifndef LCDM_H
#define LCDM_H

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LCDM_API_VERSION 1

typedef enum {
    LCDM_OK = 0,
    LCDM_ERR_INVALID = 1,      /* bad argument: null pointer, size, layout, ncol ... */
    LCDM_ERR_CUDA = 2,         /* a CUDA launch or query failed                     */
    LCDM_ERR_WORKSPACE = 3,    /* workspace missing, too small or misaligned        */
    LCDM_ERR_UNSUPPORTED = 4   /* combination not supported                         */
} lcdm_status;

enum { LCDM_FP64 = 0, LCDM_FP32_MIXED = 1 };
enum { LCDM_LAYOUT_CSR = 0, LCDM_LAYOUT_DENSE = 1, LCDM_LAYOUT_SHARED = 2 };
/* output slots (index into the out / jac / cot arrays) */
enum { LCDM_DC = 0, LCDM_T = 1, LCDM_X = 2, LCDM_DM = 3, LCDM_DL = 4, LCDM_MU = 5, LCDM_NOUT = 6 };

typedef struct {
    int32_t ncol;           /* 4 (closure), 5 (explicit Omega_k0) or 7 (+ Os, Ox) */
    int32_t precision;      /* LCDM_FP64 or LCDM_FP32_MIXED                      */
    int32_t layout;         /* LCDM_LAYOUT_*                                     */
    int32_t block;          /* threads per block (multiple of 32, <= 256); 0 = tuned */
    int32_t blocks_per_sm;  /* persistent blocks per SM; 0 = tuned               */
    int32_t lane_map;       /* pairs of a warp's range to lanes: LCDM_MAP_*      */
    int32_t deterministic;  /* 1: per-cosmology sums reproducible bit for bit (see below) */
} lcdm_opts;

/* deterministic: the per-cosmology reductions (grad of lcdm_distances_vjp,
 * loglike and grad of lcdm_gauss_loglike) add the partial sums of the warps
 * that share a row in a fixed order (a second, small kernel), instead of
 * FP64 atomics in arrival order, so that repeated calls with the same
 * inputs, launch shape and device give the same bits.  Rows owned by one
 * warp are summed in program order either way.  Needs the larger workspace
 * that lcdm_workspace_size reports for it; honoured by lcdm_distances_vjp,
 * lcdm_distances_jac, lcdm_gauss_loglike and lcdm_autotune, and refused
 * (LCDM_ERR_UNSUPPORTED) by the other entry points that reduce. */

/* lane_map: LCDM_MAP_TUNED takes the autotuner's choice for this workload
 * class, contiguous until it has run; LCDM_MAP_CONTIGUOUS gives the 32 lanes
 * 32 consecutive pairs per step (coalesced, best for unordered redshifts);
 * LCDM_MAP_INTERLEAVED gives lane l the l-th 32nd of the warp's range, so
 * that every warp sees the whole spread of z even when z is sorted within
 * the rows (every warp then runs the same code paths, which the instruction
 * cache needs). */
enum { LCDM_MAP_TUNED = 0, LCDM_MAP_CONTIGUOUS = 1, LCDM_MAP_INTERLEAVED = 2 };

/* Workspace bytes needed for B cosmologies (per-cosmology root records, and
 * with opts->deterministic the warps' partial sums). */
lcdm_status lcdm_workspace_size(int64_t B, const lcdm_opts* opts, size_t* bytes);

/* Root preparation alone (Sec. 3, eq. 3.2; App. A): roots of E^2 in z for
 * each cosmology and their derivatives with respect to the Omega columns.
 *   roots  [B][4][2] float64 (re, im): slot 0 = A, the real root with the
 *          largest |1+r| (fn15), slot 1 = B (second real root; quartic only,
 *          else -0), slots 2, 3 = the remaining pair (complex conjugates or two
 *          reals).  May be NULL.
 *   droots [B][4][2][ncol-1] float64, d root / d (Om, OL, Or[, Ok]); may be NULL.
 *   kind   [B] int32: 0 quartic 2 real + pair, 1 quartic 4 real, 2 cubic 1 real
 *          + pair, 3 cubic 3 real.  May be NULL.                               */
lcdm_status lcdm_roots(const double* params, int64_t B, const lcdm_opts* opts, double* roots,
                       double* droots, int32_t* kind, int32_t* cosmo_status, void* ws, size_t ws_bytes,
                       cudaStream_t stream);

/* Forward distances, eqs. (3.7)-(3.9) / (B.1)-(B.3) and the observables.
 *   out[LCDM_NOUT]: per-output arrays [npairs]; NULL entries are not computed
 *   (X costs most; leave it NULL when not needed).                          */
lcdm_status lcdm_distances(const double* params, int64_t B, const int64_t* offsets, const void* z,
                           int64_t n, void* const out[LCDM_NOUT], int32_t* cosmo_status,
                           const lcdm_opts* opts, void* ws, size_t ws_bytes, cudaStream_t stream);

/* Forward distances plus the per-pair Jacobian d out / d params (fused).
 *   jac[LCDM_NOUT]: per-output arrays [npairs][ncol] (column 0 = H0); NULL
 *   entries are skipped.  out may be NULL or contain NULL entries.          */
lcdm_status lcdm_distances_jac(const double* params, int64_t B, const int64_t* offsets, const void* z,
                               int64_t n, void* const out[LCDM_NOUT], void* const jac[LCDM_NOUT],
                               int32_t* cosmo_status, const lcdm_opts* opts, void* ws, size_t ws_bytes,
                               cudaStream_t stream);

/* Vector-Jacobian product fused with the forward pass (the adjoint of the
 * distance map): grad[b][c] = sum over pairs of row b and outputs o of
 * cot[o][pair] * d out_o[pair] / d params[b][c].
 *   cot[LCDM_NOUT]: cotangent arrays [npairs] (NULL = zero); out may be NULL.
 *   grad [B][ncol] float64, overwritten (NaN rows for a bad cosmo_status). */
lcdm_status lcdm_distances_vjp(const double* params, int64_t B, const int64_t* offsets, const void* z,
                               int64_t n, const void* const cot[LCDM_NOUT], void* const out[LCDM_NOUT],
                               double* grad, int32_t* cosmo_status, const lcdm_opts* opts, void* ws,
                               size_t ws_bytes, cudaStream_t stream);

/* Gaussian log-likelihood of standardised magnitudes (Sec. 4):
 *   loglike[b] = sum_i [ -(m_obs_i - mu(z_i; params_b) - M)^2 / (2 sigma^2)
 *                        - ln(sigma sqrt(2 pi)) ]
 * over the pairs of row b, and grad[b][c] = d loglike[b] / d params[b][c].
 *   m_obs indexed like z (same layout); mu_out [npairs] optional.
 *   loglike [B] float64 (required), grad [B][ncol] float64 (optional).
 * The per-row sums are accumulated in FP64.                                */
lcdm_status lcdm_gauss_loglike(const double* params, int64_t B, const int64_t* offsets, const void* z,
                               const void* m_obs, int64_t n, double M, double sigma, double* loglike,
                               double* grad, void* mu_out, int32_t* cosmo_status, const lcdm_opts* opts,
                               void* ws, size_t ws_bytes, cudaStream_t stream);

/* lcdm_gauss_loglike plus the derivative of each row's log-likelihood with
 * respect to the redshift of each of its pairs, for models whose redshifts
 * are parameters (the latent redshifts of the Sec. 4 supernova model):
 *   grad_z[i] = (m_obs_i - mu_i - M) / sigma^2 * d mu_i / d z_i,
 *   d mu / dz = (5 / ln 10) [ 1/(1+z) + S_k'(D) / (E(z) S_k(D)) ],
 * from d chi / dz = (c/H0) / E(z), the integrand of eq. (2.3) at its upper
 * limit, and the curvature map (D = chi H0 / c).
 *   grad_z [npairs] in the pass dtype (required); pairs with z = 0 get 0 (mu is
 *   -inf there); rows with a bad cosmo_status get NaN.
 *   ws: lcdm_loglike_dz_workspace_size(B, n, opts) bytes, 256-byte aligned.
 * Other arguments as lcdm_gauss_loglike.                                    */
lcdm_status lcdm_loglike_dz_workspace_size(int64_t B, int64_t n, const lcdm_opts* opts, size_t* bytes);
lcdm_status lcdm_gauss_loglike_dz(const double* params, int64_t B, const int64_t* offsets, const void* z,
                                  const void* m_obs, int64_t n, double M, double sigma, double* loglike,
                                  double* grad, void* grad_z, void* mu_out, int32_t* cosmo_status,
                                  const lcdm_opts* opts, void* ws, size_t ws_bytes, cudaStream_t stream);

/* lcdm_distances_vjp plus the derivative with respect to each pair's
 * redshift: grad_z[i] = sum_o cot[o][i] d out_o / dz_i, from the integrands
 * of eqs. (2.3)-(2.5) at the upper limit, (c/H0)/E, 1/(H0 (1+z) E) and
 * (c/H0)(1+z)^2/E, through the curvature map, d_L = (1+z) d_M and mu
 * (d mu/dz counts as 0 at z = 0).  grad_z [npairs] in the pass dtype
 * (required; for the shared layout one entry per (row, redshift) pair).
 * grad may be NULL (then only grad_z and the forward outputs are computed).
 *   ws: lcdm_loglike_dz_workspace_size(B, n, opts) bytes, 256-byte aligned.
 * Other arguments as lcdm_distances_vjp.                                   */
lcdm_status lcdm_distances_vjp_dz(const double* params, int64_t B, const int64_t* offsets, const void* z,
                                  int64_t n, const void* const cot[LCDM_NOUT], void* const out[LCDM_NOUT],
                                  double* grad, void* grad_z, int32_t* cosmo_status, const lcdm_opts* opts,
                                  void* ws, size_t ws_bytes, cudaStream_t stream);

/* Device workspace, in bytes, of lcdm_distances_vjp_host for B cosmologies
 * and n pairs (records, parameters, offsets, status, gradient, and the z,
 * cotangent and output arrays of all six outputs). */
lcdm_status lcdm_host_workspace_size(int64_t B, int64_t n, const lcdm_opts* opts, size_t* bytes);

/* lcdm_distances_vjp for data held in HOST memory: params [B][ncol],
 * offsets [B+1], z [n], cot[o] [n], out[o] [n] (out and each entry may be
 * NULL), grad [B][ncol] and cosmo_status [B] are all host arrays; CSR layout
 * only.  The paper's method is unchanged (Sec. 3); this entry point only moves
 * the data.  The batch is cut into nchunks (1..64) runs of whole rows whose
 * pair counts ramp up and down in the proportions 1 2 3 ... 3 2 1 (small
 * first and last runs: their copies are not overlapped); the host-to-device
 * copies of the next run and the device-to-host copies of the previous one
 * overlap the pair kernels of the current run.  The copies run on two streams that the library creates once
 * per device (first call); the kernels run on `stream`, after the work already
 * queued there.  Page-locked host arrays are needed for the copies to overlap.
 *   dws: device workspace of lcdm_host_workspace_size(B, n, opts) bytes,
 *        256-byte aligned.
 * The call returns when every result is in the host arrays.  Calls on one
 * device share the internal streams: they must not run concurrently from
 * several host threads.                                                     */
lcdm_status lcdm_distances_vjp_host(const double* params, int64_t B, const int64_t* offsets, const void* z,
                                    int64_t n, const void* const cot[LCDM_NOUT], void* const out[LCDM_NOUT],
                                    double* grad, int32_t* cosmo_status, const lcdm_opts* opts, void* dws,
                                    size_t dws_bytes, int32_t nchunks, cudaStream_t stream);

/* Largest B accepted by lcdm_distances_static. */
#define LCDM_STATIC_MAX_COSMOLOGIES 4096

/* lcdm_distances without a workspace argument, for callers that cannot
 * allocate device memory: for example a caller that is capturing a CUDA
 * graph (where cudaMalloc is not allowed), one that runs under a fixed memory
 * budget with no allocator of its own, or plain C code that has no device
 * allocator at hand.  (The paper has no counterpart; this is a convenience of
 * this library.)
 *   Scratch lives in a fixed device array inside the library, sized for
 *   LCDM_STATIC_MAX_COSMOLOGIES cosmologies (about 6 MB), which stays
 *   allocated on every device that loads the library until the process exits.
 *   B larger than that is rejected with LCDM_ERR_INVALID; nothing is enqueued.
 *   The function calls no cudaMalloc, cudaFree or other allocating routine.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress); make that first call outside any stream capture.
 *   Every call on a device shares the one array and overwrites it fully, so
 *   calls whose kernels may overlap on the GPU (other streams, other host
 *   threads) race: order them on one stream or serialise them.
 *   Other arguments, outputs and status codes as lcdm_distances.           */
lcdm_status lcdm_distances_static(const double* params, int64_t B, const int64_t* offsets, const void* z,
                                  int64_t n, void* const out[LCDM_NOUT], int32_t* cosmo_status,
                                  const lcdm_opts* opts, cudaStream_t stream);

/* Times the candidate launch shapes (threads per block x persistent blocks
 * per SM x lane map) of the pair kernel on the given inputs, keeps the
 * fastest in a process-wide cache keyed by (precision, outputs, tangents,
 * layout, log2 npairs) and returns it.  Arguments as lcdm_distances_vjp (grad
 * NULL selects a forward-only shape and cot is then ignored; out entries are
 * overwritten).  The call synchronises the stream; do not call it while
 * capturing a CUDA graph.                                                   */
lcdm_status lcdm_autotune(const double* params, int64_t B, const int64_t* offsets, const void* z, int64_t n,
                          const void* const cot[LCDM_NOUT], void* const out[LCDM_NOUT], double* grad,
                          int32_t* cosmo_status, const lcdm_opts* opts, void* ws, size_t ws_bytes,
                          cudaStream_t stream, int32_t* best_block, int32_t* best_blocks_per_sm,
                          float* best_ms, int32_t* best_lane_map);

/* ---------------------------------------------------------------------------
 * General limits.  Eqs. (2.3)-(2.5) are integrals from z1 to z2; the entry
 * points above take z1 = 0.  The two below take a lower limit z1[b] >= 0 per
 * row (device, float64).  They evaluate eqs. (3.7)-(3.9) / (B.1)-(B.3) with
 * X_m = sqrt(z2 - r_m), Y_m = sqrt(z1 - r_m), Delta z = z2 - z1 (Sec. 3.1) in
 * the form they take in the coordinate of an observer at z1: with s = 1 + z1
 * and E1 = E^2(z1), the row becomes the closed cosmology
 *   (H0 sqrt(E1), Om s^3/E1, OL/E1, Or s^4/E1), Ok' = Ok s^2/E1 by closure,
 * with roots (r - z1)/s, the pair's upper limit becomes (z2 - z1)/s, and
 * every output is the z1 = 0 result of that cosmology times a power of s.
 * The root preparation therefore runs once per row (on the shifted
 * parameters) and cosmo_status refers to the shifted cosmology: status 1 means
 * a real root of E^2 at z >= z1; status 2 also covers z1 < 0, non-finite z1
 * or E^2(z1) <= 0.
 * ------------------------------------------------------------------------- */

/* Workspace bytes of lcdm_distances_between (B rows, n as in the layout) and
 * of lcdm_limits (n = 0).                                                   */
lcdm_status lcdm_between_workspace_size(int64_t B, int64_t n, const lcdm_opts* opts, size_t* bytes);

/* Distances between z1[b] and each pair's z2 (layouts LCDM_LAYOUT_CSR and
 * LCDM_LAYOUT_DENSE; SHARED is rejected), with the fused adjoint when grad is
 * not NULL.  Per pair, in the output slots of the z1 = 0 entry points:
 *   LCDM_DC  chi(z1, z2)                        eq. (2.3), via (3.7)/(B.1)
 *   LCDM_T   t(z1, z2)                          eq. (2.4), via (3.8)/(B.2)
 *   LCDM_X   d_abs(z1, z2)                      eq. (2.5), via (3.9)/(B.3)
 *   LCDM_DM  transverse comoving distance S_k(chi(z1, z2)), today's units
 *   LCDM_DL  (1+z2) d_M / (1+z1)^2: the luminosity distance of a source at
 *            z2 seen by a comoving observer at z1 (its redshift relative to
 *            that observer is (1+z2)/(1+z1) - 1)
 *   LCDM_MU  5 log10(d_L / 10 pc)
 * With z1 = 0 these are the outputs of lcdm_distances.  Domain z2 >= z1:
 * pairs with z2 < z1 give NaN outputs and add nothing to the gradient; z2 = z1
 * gives 0 (mu = -inf).
 *   cot, grad: as lcdm_distances_vjp (cot required when grad is not NULL;
 *   grad NULL computes the forward outputs only).  out may be NULL when grad
 *   is not, and its entries may be NULL.
 *   ws: lcdm_between_workspace_size(B, n, opts) bytes, 256-byte aligned.
 * Precision, units, streams and errors as above.                            */
lcdm_status lcdm_distances_between(const double* params, int64_t B, const double* z1, const int64_t* offsets,
                                   const void* z2, int64_t n, const void* const cot[LCDM_NOUT],
                                   void* const out[LCDM_NOUT], double* grad, int32_t* cosmo_status,
                                   const lcdm_opts* opts, void* ws, size_t ws_bytes, cudaStream_t stream);

/* The upper limit at infinity, per row (Sec. 2.1.1: the age of the universe
 * at z1 is t(z1, inf)):
 *   chi_inf [B]  chi(z1, inf) [Mpc], the comoving distance to the particle
 *                horizon (limit of eq. 3.7 / B.1)
 *   t_inf   [B]  t(z1, inf) [Gyr], the age at redshift z1 (limit of eq. 3.8 /
 *                B.2); at z1 = 0 the present age of the universe
 * (d_abs diverges).  Either may be NULL.  Always FP64 (float64 arrays,
 * whatever opts->precision).  With grad not NULL, grad[b][c] =
 * cot_chi[b] d chi_inf / d params[b][c] + cot_t[b] d t_inf / d params[b][c]
 * (a NULL cotangent counts as zero).  opts->layout is ignored.
 *   ws: lcdm_between_workspace_size(B, 0, opts) bytes, 256-byte aligned.    */
lcdm_status lcdm_limits(const double* params, int64_t B, const double* z1, double* chi_inf, double* t_inf,
                        const double* cot_chi, const double* cot_t, double* grad, int32_t* cosmo_status,
                        const lcdm_opts* opts, void* ws, size_t ws_bytes, cudaStream_t stream);

/* Human-readable name of a lcdm_status value (static string). */
const char* lcdm_status_string(int status);

/* Number of kernels this library has launched in this process so far. */
int64_t lcdm_launch_count(void);

/* Issue-rate probes (no counterpart in the paper): the denominators of a
 * roofline for the pair kernel, measured on the GPU at hand.  what = 0: FP32
 * fused multiply-add; 1: FP32 reciprocal square root (the special-function
 * unit that also serves division and square root); 2: FP64 fused
 * multiply-add.  Launches blocks x threads threads (threads a multiple of 32,
 * <= 1024), each running lcdm_probe_ops_per_thread(iters) operations of that
 * kind in 8 independent chains, and writes one value per thread to out
 * (device, blocks * threads floats, or doubles for what = 2).  Time the call
 * with events on `stream`; rate = blocks * threads * ops / time.  Returns
 * LCDM_ERR_INVALID for a bad shape or kind, before any launch. */
int64_t lcdm_probe_ops_per_thread(int32_t iters);
lcdm_status lcdm_probe(int32_t what, void* out, int32_t blocks, int32_t threads, int32_t iters,
                       cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* LCDM_H */
