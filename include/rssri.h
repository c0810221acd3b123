/*
 * rssri.h - C ABI of the GB300 (sm_103a) range-separated stochastic-RI GF2
 * self-energy library, librssri.so.
 *
 * The library evaluates, on one GPU, the second-order (GF2) self-energy
 * Sigma(tau) on an imaginary-time grid and the correlation energy per
 * electron, with the electron-repulsion integrals split into a large part
 * treated by deterministic RI and a remainder treated by stochastic RI
 * (Dou, Chen, Takeshita, Baer, Neuhauser, Rabani, arXiv:2005.12338):
 *
 *   Sec. II, Eqs. 4-8    RI factorisation, K^Q_ij = sum_A (ij|A) V^{-1/2}_AQ
 *   Sec. II, Eqs. 9-10   stochastic RI, R^xi_ij = sum_A (ij|A)(V^{-1/2} theta^xi)_A
 *   Sec. II, Eqs. 11-16  range separation: (ij|A)^L screen, [K^Q]^L and its
 *                        cut, R^L = [K]^L theta, R^S = R - R^L
 *   Sec. III, Eq. 17     the imaginary-time Green's function G(tau)
 *   Sec. III, Eq. 20/25  the GF2 self-energy and its RS-SRI form
 *   Sec. IV, Eq. 26      E_corr = (1/N_e) int_0^beta Tr[Sigma(tau) G(beta-tau)]
 *
 * Conventions shared by every entry point
 *   - All floating point is IEEE binary64 (double).
 *   - Arrays are dense, row-major (C order), with the shapes stated below.
 *   - Pointers are caller-owned.  The library never frees them and keeps no
 *     reference to them after the call returns, except that rssri_setup()
 *     copies the problem into handle-owned device memory.
 *   - Every call returns an rssri_status (0 = success, negative = error) and
 *     never throws.  On error nothing is written to the outputs except where
 *     stated; the handle stays usable unless the code is RSSRI_ERR_CUDA.
 *   - All device work is issued on the handle's stream; calls returning host
 *     scalars synchronise that stream before they return.
 *   - One handle per host thread at a time.  Handles do not share state.
 *   - Results are deterministic: the same inputs, options and seed on the same
 *     GPU give bitwise-identical outputs (fixed-order reductions, no
 *     floating-point atomics).
 */
#ifndef RSSRI_H
#define RSSRI_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RSSRI_API __attribute__((visibility("default")))
#else
#define RSSRI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------- status codes */
typedef enum {
  RSSRI_OK = 0,
  RSSRI_ERR_INVALID_ARG = -1,     /* a size, threshold, pointer or option is out of range */
  RSSRI_ERR_NOT_SPD = -2,         /* metric V is not symmetric positive definite (the
                                     inverse-square-root iteration did not converge)  */
  RSSRI_ERR_NONSYMMETRIC_ERI = -3,/* (ij|A) != (ji|A) for some i, j, A                */
  RSSRI_ERR_OOM = -4,             /* device allocation failed                          */
  RSSRI_ERR_CUDA = -5,            /* a CUDA runtime call failed; handle is unusable    */
  RSSRI_ERR_TIMEOUT = -6,         /* a bounded device-side wait expired                */
  RSSRI_ERR_NOT_READY = -7,       /* rssri_sigma before a successful rssri_setup       */
  RSSRI_ERR_NONFINITE = -8,       /* an input or result is NaN or infinite             */
  RSSRI_ERR_RANGE = -9            /* a double-float input (RSSRI_PREC_DF64 or
                                     RSSRI_DD_DF64) has its largest magnitude outside
                                     [2^-40, 2^40], where fp32 pairs lose precision;
                                     use IEEE fp64 or RSSRI_DD_OZ instead           */
} rssri_status;

/* Where the arrays of a call live. */
enum { RSSRI_PTR_DEVICE = 0, RSSRI_PTR_HOST = 1 };

/* Estimator.  RSSRI_EST_CV (default): Sigma = Sigma_DD + (1/N_s) sum_xi
 * [F(R^xi, R'^xi) - F(R^Lxi, R'^Lxi)], where F(X, Y) is Eq. 20 evaluated on
 * the rank-one integrals X(x)X and Y(x)Y and Sigma_DD is Eq. 20 on
 * v^L = sum_Q [K^Q]^L [K^Q]^L; every bracket of Eq. 25 equals
 * D + <R R> - <R^L R^L>, and this form keeps D D exact while pairing sample
 * xi of theta with sample xi of theta'.
 * RSSRI_EST_SRI: [K]^L is taken as empty, which is the plain stochastic RI of
 * Eq. 10 (the eps -> 1 limit of Sec. II).
 * RSSRI_EST_LITERAL: Eq. 25 with the product of brackets expanded term by
 * term, D exact inside every bracket: Sigma = Sigma_DD + Phi(D, S'_xi) +
 * Phi(S_xi, D) + Phi(S_xi, S'_xi) averaged over xi, S_xi = R(x)R - R^L(x)R^L.
 * The cross terms with D are built per sample from the pair-space v^L
 * (exchange) and from [K]^L (direct), about 4 N_aux P + 8 P^2 flops per
 * (pair, tau) unit on top of four chains; fp64 chain only. */
enum { RSSRI_EST_CV = 0, RSSRI_EST_SRI = 1, RSSRI_EST_LITERAL = 2 };

/* Arithmetic of the chain products of the stochastic part (S8).
 * RSSRI_PREC_FP64: every product in fp64 (the plain form).
 * RSSRI_PREC_BF16: the chain is evaluated in the range-separated split of
 *   Eqs. 14-15 (C^L = R^L G R'^L, dC = R^S G R' + R^L G R'^S, so that the
 *   difference F(R,R') - F(R^L,R'^L) is formed from small terms only) with
 *   bf16 operands and fp32 accumulation on the tensor cores; V^{-1/2}, the
 *   deterministic block, traces and energies stay fp64.  Needs N >= 16 and a
 *   GPU with tcgen05 (sm_100 family); its error is of relative order 1e-3 of
 *   the stochastic remainder Sigma - Sigma_DD.
 * RSSRI_PREC_TF32: the same split with operands rounded to tf32 (10 stored
 *   mantissa bits, kept in fp32 storage) and fp32 accumulation: about 8x
 *   smaller operand rounding than bf16 at twice the operand bytes and half
 *   the tensor-core rate.
 * RSSRI_PREC_DF64: the plain form's products in double-float arithmetic on
 *   the fp32 pipes (each fp64 value as a pair of floats, error-free products
 *   and sums, ~1e-13 relative): fp64-accurate, within the same 1e-10 of the
 *   fp64 form, and several times faster on GPUs whose fp64 rate is a small
 *   fraction of their fp32 rate.  A pair has fp32's exponent range: every
 *   input matrix converted to pairs ((ij|A), the metric's Newton-Schulz
 *   iterates, [K]^L and v^L, the sign vectors and factors, and G and
 *   G(beta - tau) per tau point) must have its largest magnitude in
 *   [2^-40, 2^40], else the call returns RSSRI_ERR_RANGE.  Intermediates of
 *   the block (Gamma, T) are not checked: they are products of checked
 *   inputs and, for G with entries far below 2^-40 at some tau, lose
 *   precision without notice; IEEE fp64 and RSSRI_DD_OZ keep fp64's range. */
enum { RSSRI_PREC_FP64 = 0, RSSRI_PREC_BF16 = 1, RSSRI_PREC_TF32 = 2, RSSRI_PREC_DF64 = 3 };

typedef struct rssri_handle rssri_handle;

/* The problem (Sec. II-III).
 *   n       number of basis functions N            (1 <= n <= 4096)
 *   n_occ   occupied orbitals, N_e = 2 n_occ       (1 <= n_occ <= n-1)
 *   n_aux   auxiliary functions N_aux              (1 <= n_aux < 2^20)
 *   n_tau   imaginary-time points                  (n_tau >= 1)
 *   eri3    [n][n][n_aux]  (ij|A) of Eq. 5; must satisfy (ij|A) == (ji|A) exactly
 *   metric  [n_aux][n_aux] V_AB of Eq. 6; symmetric positive definite
 *   orb_e   [n]            orbital energies, the first n_occ occupied
 *   orb_c   [n][n]         AO x MO coefficients, orthonormal (C^T C = I, S = I)
 *   tau     [n_tau]        grid nodes, each in (0, beta)
 *   tau_w   [n_tau]        quadrature weights of Eq. 26's tau integral
 *   mu      chemical potential; beta inverse temperature (finite, > 0)
 *   ptr_kind RSSRI_PTR_DEVICE or RSSRI_PTR_HOST, for all arrays above
 * G is the zero-temperature non-interacting Green's function of the given
 * orbitals (Eq. 17 with occupations 1 and 0):
 *   G(tau) = -C_v exp(-(e_v - mu) tau) C_v^T,
 *   G(beta - tau) = -C_o exp((e_o - mu) tau) C_o^T. */
typedef struct {
  int32_t n, n_occ, n_aux, n_tau;
  int32_t ptr_kind;
  int32_t reserved0;
  const double *eri3;
  const double *metric;
  const double *orb_e;
  const double *orb_c;
  const double *tau;
  const double *tau_w;
  double mu, beta;
} rssri_problem;

/* Options.
 *   eps_prime  epsilon' of Eq. 11, in [0, 1]: (ij|A) is kept when
 *              |(ij|A)| >= (eps'/N) min(M_i, M_j), M_j = max_{i,A} |(ij|A)|
 *              (the paper's per-j maximum, applied symmetrically).
 *   eps        epsilon of Eq. 13, in [0, 1]: [K^Q_ij]^L is kept when
 *              |[K^Q_ij]^L| >= eps * max |[K]^L| (global maximum).
 *   n_s        number of stochastic sample pairs (theta^xi, theta'^xi), >= 2.
 *   seed       64-bit seed of the counter-based Rademacher draws: theta^xi_Q
 *              of set s (0: theta, 1: theta') is -1 when bit 63 of the first
 *              SplitMix64 output from state seed XOR (s 2^60 + xi 2^20 + Q) is
 *              set, else +1 (SplitMix64: Steele, Lea and Flood, OOPSLA 2014).
 *   xi_offset  first sample index (resume: runs over [xi_offset, xi_offset+n_s)
 *              concatenate exactly), xi_offset + n_s < 2^40.
 *   estimator  RSSRI_EST_CV, RSSRI_EST_SRI or RSSRI_EST_LITERAL (the last
 *              with precision RSSRI_PREC_FP64 and cv = 0).
 *   precision  RSSRI_PREC_FP64, RSSRI_PREC_BF16, RSSRI_PREC_TF32 or
 *              RSSRI_PREC_DF64 (chain products only).
 *   pair_batch sample pairs processed per group of launches (0 = all;
 *              fp64 and double-float chains; the tensor-core chains take all
 *              pairs at once).
 *   profile    1: time every kernel class with CUDA events on the handle's
 *              stream (rssri_stats.prof_*); 0: off.
 *   cv         1: weight the large-part control variate element-wise by the
 *              coefficients c_ij(tau) of the network trained by
 *              rssri_cv_train (RSSRI_EST_CV only; with the tensor-core
 *              chains, F(R^L, R'^L) of every pair is formed by one more
 *              product on the tensor cores); 0: c = 1.
 *   dd_arith   arithmetic of the deterministic block (its products and
 *              exchange contraction): RSSRI_DD_FP64 (IEEE fp64 FMAs),
 *              RSSRI_DD_DF64 (double-float: each fp64 value as a pair of
 *              floats, error-free products and sums on the fp32 pipes, ~1e-13
 *              relative; values must stay inside fp32's exponent range, about
 *              1e-38 to 3e38, or lose their relative precision), or
 *              RSSRI_DD_OZ (fp64-accurate sliced products on the bf16 tensor
 *              cores: each row of an fp64 operand is scaled by a power of two
 *              and split into six 8-bit digits, every digit product and the
 *              accumulation of the leading levels are exact, ~1e-12 of
 *              sum |a||b| per dot product, with fp64's exponent range; the
 *              segmented product K^Q G runs in double-float on G(tau)
 *              normalised by a power of two per tau point and rescaled
 *              exactly, the block being homogeneous of degree 2 in G).  RSSRI_DD_OZ
 *              needs a GPU with tcgen05 (sm_100 family); its R, R^L and
 *              v^L are formed as for RSSRI_DD_DF64.
 *              The value given to rssri_setup sets how v^L and
 *              the cached block are formed; the value given to
 *              rssri_sigma_from_g sets the arithmetic of its rebuilt block,
 *              and that given to rssri_sigma the arithmetic of R, R^L and of
 *              the literal estimator's exchange builds. */
typedef struct {
  double eps_prime, eps;
  int64_t n_s;
  uint64_t seed;
  int64_t xi_offset;
  int32_t estimator;
  int32_t precision;
  int64_t pair_batch;
  int32_t profile;
  int32_t dd_arith;
  int32_t cv;         /* 1: apply the learned control variate (see rssri_cv_train) */
  int32_t test_wait_polls;  /* testing only, 0 otherwise: > 0 makes the tensor-core
                               kernels of this call issue no copy or product and give
                               up each bounded wait after this many polls, so that the
                               call returns RSSRI_ERR_TIMEOUT with nothing in flight */
  int32_t test_fail_alloc;  /* testing only, 0 otherwise: k > 0 makes the k-th device
                               allocation of this call fail (RSSRI_ERR_OOM) without
                               calling the allocator */
  int32_t reserved0;
} rssri_options;

enum { RSSRI_DD_FP64 = 0, RSSRI_DD_DF64 = 1, RSSRI_DD_OZ = 2 };

/* Kernel classes of the per-class profile (rssri_stats.prof_*). */
enum {
  RSSRI_PROF_CHAIN_GEMM = 0,  /* S8 chain products X G, (X G) Y, C Gb, (2 t I - B) C */
  RSSRI_PROF_DD_SPMM = 1,     /* S7 exchange term, pair-space contraction         */
  RSSRI_PROF_DD_GEMM = 2,     /* S7 other products                                */
  RSSRI_PROF_FACTOR_GEMM = 3, /* S4/S5 theta W, R, R^L                             */
  RSSRI_PROF_SETUP_GEMM = 4,  /* S1/S3 Newton-Schulz, [K]^L, D                     */
  RSSRI_PROF_GREEN = 5,       /* S6                                               */
  RSSRI_PROF_OTHER = 6,       /* screening, compaction, cuts, folds, reductions   */
  RSSRI_PROF_SLICE = 7,       /* digit slicing of the operands of RSSRI_DD_OZ      */
  RSSRI_PROF_NCLASS = 8
};

/* Counters of the last setup / sigma call. */
typedef struct {
  int64_t n_pairs_screened; /* (i,j) pairs with >= 1 kept (ij|A), Eq. 11        */
  int64_t nnz_eri_l;        /* kept (ij|A) elements, Eq. 11                     */
  int64_t n_pairs_large;    /* (i,j) pairs with a non-zero [K]^L row, Eq. 13     */
  int64_t nnz_k_l;          /* non-zero [K^Q_ij]^L elements after the cut        */
  double k_l_max;           /* max |[K^Q_ij]^L| before the cut                   */
  int32_t metric_iterations;/* Newton-Schulz iterations used for V^{-1/2}       */
  int32_t reserved0;
  double metric_residual;   /* max |Z Y - I| at exit (Z ~ V^{-1/2}, Y ~ V^{1/2}) */
  double e_dd;              /* Eq. 26 for the deterministic block alone          */
  double e_corr;            /* Eq. 26 for the full estimate                      */
  double e_stderr;          /* sample std of the per-pair energies / sqrt(n_s)   */
  double t_setup_ms;        /* device time of rssri_setup (S1-S3, S6, S7)        */
  double t_green_dd_ms;     /* device time of G(tau) and Sigma_DD(tau) in the last
                               sampling call (0 when it reused the setup's)     */
  double t_sample_ms;       /* device time of theta, R, chains, energy, output   */
  int64_t kernel_launches;  /* kernels launched by the last setup + sigma        */
  int64_t prof_launches[RSSRI_PROF_NCLASS]; /* per class, last setup + sigma      */
  double prof_ms[RSSRI_PROF_NCLASS];    /* device ms per class (profile = 1)     */
  double prof_gflop[RSSRI_PROF_NCLASS]; /* algorithmic fp64 GFLOP per class: 2mnk
                                           per product, 2 N_aux P^2 per S7 exchange
                                           contraction (P kept pairs)            */
  double prof_tensor_gflop[RSSRI_PROF_NCLASS]; /* GFLOP issued to the tensor cores
                                           per class (digit products of the sliced
                                           block and bf16/tf32 chain products, over
                                           the padded tiles actually computed)   */
  double t_cv_c_ms;         /* device time of the learned control variate's
                               coefficients c in the last sampling call (0 when it
                               reused them: c is computed once per setup, caller G
                               and parameter set; included in t_sample_ms)      */
} rssri_stats;

/* ------------------------------------------------------------- lifetime */

/* Create a handle bound to CUDA device `device` and stream `stream` (a
 * cudaStream_t passed as void*; NULL = the legacy default stream).  The
 * handle owns all scratch device memory; nothing is allocated until
 * rssri_setup(). */
RSSRI_API int rssri_create(rssri_handle **out, int device, void *stream);

/* Free the handle and its device memory.  NULL is accepted. */
RSSRI_API void rssri_destroy(rssri_handle *h);

/* Static description of a status code. */
RSSRI_API const char *rssri_status_string(int code);

/* Name of the last CUDA runtime error that made a call of this thread return
 * RSSRI_ERR_CUDA or RSSRI_ERR_OOM (cudaGetErrorName), or "" if none has;
 * for diagnostics.  The string is static. */
RSSRI_API const char *rssri_last_cuda_error(void);

/* ----------------------------------------------------------- the path */

/* Steps that depend only on the system, the thresholds and G:
 *   S1  W = V^{-1/2} (Eq. 7) by the coupled Newton-Schulz iteration (fp64);
 *   S2  screen (ij|A) with eps' (Eq. 11) and compact the kept (i,j) pairs;
 *   S3  [K]^L = (ij|A)^L W on the kept pairs (Eq. 12), cut at eps (Eq. 13),
 *       and the pair-space product D = [K]^L [K]^L^T used by the exchange
 *       part of the deterministic block;
 *   S6  G(tau), G(beta - tau) (Eq. 17) for every tau of the grid;
 *   S7  Sigma_DD(tau): Eq. 20 on v^L = sum_Q [K^Q]^L [K^Q]^L (the terms of
 *       Eq. 25 that hold no stochastic factor), in the arithmetic o->dd_arith.
 * S6 and S7 do not depend on the draws: their results stay in the handle and
 * every rssri_sigma call on this setup reuses them (rssri_stats.t_green_dd_ms
 * is then 0).  Copies the problem into handle-owned device memory when it is
 * given in host memory; device arrays are referenced until the next setup.
 * Errors: INVALID_ARG (sizes, thresholds, dd_arith, null pointers, tau outside
 * (0, beta)), NONSYMMETRIC_ERI, NOT_SPD, NONFINITE, OOM, CUDA. */
RSSRI_API int rssri_setup(rssri_handle *h, const rssri_problem *p, const rssri_options *o);

/* Steps that depend on the sample draws, for every tau of the grid:
 *   S4  theta, theta' (Rademacher) and u = W theta;
 *   S5  R = (ij|A) u (Eq. 9), R^L = [K]^L theta (Eq. 14);
 *   S8  per sample pair and factor pair (X, Y): C = X G Y, t = Tr(C Gb),
 *       B = C Gb, accumulate (2 t C - B C) with weight +-1/N_s (Eq. 25);
 *   S9  E_corr (Eq. 26, sign taken so that a Hartree-Fock G gives the MP2
 *       energy per electron: E_corr = -(1/N_e) sum_tau w_tau Tr[Sigma Gb]),
 *       per-pair energies and their standard error;
 *   S10 sigma = (Sigma + Sigma^T)/2,
 * on top of the G(tau) and Sigma_DD(tau) of the setup (S6, S7).  If the last
 * call on the handle was rssri_sigma_from_g, S6 and S7 are first rebuilt for
 * the orbitals' G with the setup's dd_arith.
 * Outputs (kind per the problem's ptr_kind):
 *   sigma   [n_tau][n][n]  overwritten
 *   e_pair  [n_s] per-pair estimates of E_corr (their mean is E_corr), or NULL
 *   e_corr, e_stderr       host scalars, either may be NULL
 *   st      host stats, may be NULL
 * o->eps_prime and o->eps are ignored here: the split made by rssri_setup
 * is used.  Errors: NOT_READY, INVALID_ARG, NONFINITE, OOM, CUDA, TIMEOUT. */
RSSRI_API int rssri_sigma(rssri_handle *h, const rssri_options *o, double *sigma,
                double *e_pair, double *e_corr, double *e_stderr,
                rssri_stats *st);

/* As rssri_sigma, but with G(tau) and G(beta - tau) supplied by the caller
 * (the paper's general, e.g. self-consistent, G of Eq. 17) instead of being
 * built from the orbitals: g and gb are [n_tau][n][n], each matrix symmetric,
 * of the problem's ptr_kind.  The deterministic block (S7) is rebuilt for
 * this G in the arithmetic o->dd_arith on every call. */
RSSRI_API int rssri_sigma_from_g(rssri_handle *h, const rssri_options *o,
                       const double *g, const double *gb, double *sigma,
                       double *e_pair, double *e_corr, double *e_stderr,
                       rssri_stats *st);

/* Asynchronous form of rssri_sigma: enqueues the same work on the handle's
 * stream and returns without waiting for it.  sigma (required) and e_pair
 * (optional) must stay valid until rssri_sigma_wait returns; host arrays are
 * copied asynchronously only if they are pinned.  At most one call may be
 * pending per handle; until it has been waited for, the handle accepts no
 * other call except rssri_destroy (which waits).  The energies, statistics
 * and any error of the enqueued work are returned by rssri_sigma_wait. */
RSSRI_API int rssri_sigma_async(rssri_handle *h, const rssri_options *o, double *sigma,
                                double *e_pair);
RSSRI_API int rssri_sigma_wait(rssri_handle *h, double *e_corr, double *e_stderr,
                               rssri_stats *st);

/* Many independent systems at once: rssri_sigma on count distinct handles
 * (each set up beforehand, each on its own stream so that their work can
 * overlap on the device) with the same options.  All calls are enqueued
 * before any is waited for.  sigma[i], e_pair[i] (e_pair may be NULL),
 * e_corr[i] and e_stderr[i] (either may be NULL) belong to hs[i].  Returns
 * the first error; every call that was enqueued is waited for. */
RSSRI_API int rssri_sigma_batch(rssri_handle *const *hs, int count, const rssri_options *o,
                                double *const *sigma, double *const *e_pair, double *e_corr,
                                double *e_stderr);

/* ------------------------------------------------------- intermediates */

/* Intermediates kept on the device after setup / sigma, for inspection. */
typedef enum {
  RSSRI_BUF_W = 0,          /* [n_aux][n_aux]       V^{-1/2}                           */
  RSSRI_BUF_COLMAX = 1,     /* [n]                  M_j of Eq. 11                     */
  RSSRI_BUF_ERI_L = 2,      /* [n][n][n_aux]        (ij|A)^L, zero where screened out */
  RSSRI_BUF_K_L = 3,        /* [n][n][n_aux]        [K^Q_ij]^L after the cut          */
  RSSRI_BUF_THETA = 4,      /* [2][n_s][n_aux]      theta, theta' as +-1.0            */
  RSSRI_BUF_R = 5,          /* [2][n_s][n][n]       R for theta, theta'               */
  RSSRI_BUF_R_L = 6,        /* [2][n_s][n][n]       R^L for theta, theta'             */
  RSSRI_BUF_G = 7,          /* [n_tau][n][n]        G(tau)                            */
  RSSRI_BUF_GB = 8,         /* [n_tau][n][n]        G(beta - tau)                     */
  RSSRI_BUF_SIGMA_DD = 9,   /* [n_tau][n][n]        deterministic block               */
  RSSRI_BUF_SIGMA_RAW = 10, /* [n_tau][n][n]        Sigma before symmetrisation       */
  RSSRI_BUF_CV_PARAMS = 11, /* [RSSRI_CV_NPARAM] float: network parameters             */
  RSSRI_BUF_CV_C = 12       /* [n_tau][n][n]        coefficients c of the last cv run   */
} rssri_buffer;

/* Size in bytes of an intermediate (0 if it does not exist yet). */
RSSRI_API int rssri_buffer_bytes(rssri_handle *h, int which, size_t *bytes);

/* Copy an intermediate to `dst` (device or host per dst_kind); `bytes` must
 * equal rssri_buffer_bytes().  Synchronises the handle's stream. */
RSSRI_API int rssri_export(rssri_handle *h, int which, void *dst, size_t bytes, int dst_kind);

/* ------------------------------------------- learned control variate */

/* The large part of Eq. 25 is a control variate with an exactly known mean:
 * for independent theta, theta', E[F(R^L, R'^L)] = Sigma_DD.  So for any
 * coefficients c_ij(tau) fixed independently of the draws they are used with,
 *   Sigma_c = mean_xi F(R, R') - c o (mean_xi F(R^L, R'^L) - Sigma_DD)
 * is unbiased (c = 1 is the default estimator), and per element its variance
 * is smallest at c* = Cov(F, F^L) / Var(F^L).  A network maps features of
 * (i, j, tau) to c: |i-j|/N, ln tau / ln beta, Sigma_DD_ij / max|Sigma_DD|,
 * G_ii, G_jj, Gb_ii, Gb_jj (each over its largest diagonal magnitude), the
 * norms of rows i and j of [K]^L over their largest, [i == j]; layers
 * 10 -> 256 -> 256 -> 256 -> 1 with SiLU, c = 1 + output; fp32.
 * Parameter layout (floats): W0[256][10] b0[256] W1[256][256] b1[256]
 * W2[256][256] b2[256] W3[1][256] b3[1]. */
#define RSSRI_CV_NPARAM 134657

/* Train the network on an independent run: evaluates the chain with options
 * `o` (precision FP64 or DF64, estimator CV; use a seed not used for the
 * estimates), collects per-element sums of F, F^L and their products, forms
 * the targets c* and weights Var(F^L), and runs `steps` Adam steps (learning
 * rate lr, betas 0.9/0.999) on minibatches of `batch` elements, minimising
 * sum w (c - c*)^2 / sum w, on the GPU.  init_params: host, RSSRI_CV_NPARAM
 * floats.  loss_before/after (host, may be NULL): that loss at init_params and
 * after training, over the first 65536 elements in a fixed order.
 * Errors: NOT_READY, INVALID_ARG, OOM, CUDA. */
RSSRI_API int rssri_cv_train(rssri_handle *h, const rssri_options *o, const float *init_params,
                             int steps, int batch, float lr, double *loss_before,
                             double *loss_after);

/* Load network parameters (host, RSSRI_CV_NPARAM floats) instead of training;
 * they are used by rssri_sigma with options.cv = 1. */
RSSRI_API int rssri_cv_set_params(rssri_handle *h, const float *params);

/* The training loss and its gradient for given parameters and data (all host
 * arrays): x [m][10] features, target [m], weight [m], params
 * [RSSRI_CV_NPARAM]; writes loss (1 float) and grad [RSSRI_CV_NPARAM].
 * Evaluated by the same GPU kernels that train the network. */
RSSRI_API int rssri_cv_loss_grad(rssri_handle *h, const float *x, const float *target,
                                 const float *weight, int m, const float *params, float *loss,
                                 float *grad);

/* ---------------------------------------------------- allocation-free */

/* Capacity, in tau points, of the fixed scratch of rssri_energy_static. */
#define RSSRI_STATIC_MAX_TAU 4096

/* The paper has no counterpart to this entry point; it exists for callers
 * that may not allocate device memory: code that runs while a stream is being
 * captured into a CUDA graph (an allocation there invalidates the capture),
 * hosts whose pool allocator owns all device memory and forbids libraries
 * from allocating, and loops that must never wait on the allocator.
 *
 * It evaluates E_corr = -(1/N_e) sum_t tau_w[t] Tr[sigma[t] gb[t]] (Eq. 26,
 * N_e = 2 n_occ, same sign and same summation order as rssri_sigma) for a
 * self-energy the caller already holds, with no handle and no allocation.
 *   sigma  device, [n_tau][n][n]  Sigma(tau)
 *   gb     device, [n_tau][n][n]  G(beta - tau)
 *   tau_w  device, [n_tau]        quadrature weights
 *   e_corr device, [1]            output, written on `stream`
 *   stream cudaStream_t as void* (NULL = legacy default stream)
 * Its scratch is a static device array of RSSRI_STATIC_MAX_TAU doubles
 * (32 KiB), present on every GPU that loads the library until the process
 * exits.  The first call on each device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make that first call before
 * any stream capture.  All calls share the array: calls whose work overlaps on
 * the GPU (different streams, or concurrent host threads) race on it and must
 * be serialised by the caller.  Returns RSSRI_ERR_INVALID_ARG for null
 * pointers, n outside [1, 4096], n_occ < 1 or n_tau outside
 * [1, RSSRI_STATIC_MAX_TAU]; RSSRI_ERR_CUDA if a launch fails.  Does not
 * synchronise. */
RSSRI_API int rssri_energy_static(const double *sigma, const double *gb, const double *tau_w,
                                  int n, int n_tau, int n_occ, double *e_corr, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RSSRI_H */
