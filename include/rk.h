/*
 * rk.h -- C ABI of librk: rapid approximate Kriging prediction on one GPU.
 *
 * The library implements the rapid predictor of "Rapid Approximation
 * Prediction for Kriging" (Li, Fasshauer, Nychka), Section 2: the covariance
 * between a grid node and an off-grid site is replaced by a local
 * interpolation of grid covariances (Eqs. 6-7, weights of Eq. "weights"), so
 * that prediction becomes a sparse scatter c* = A^T c followed by a discrete
 * convolution of c* with the Matern filter on the grid (Eqs. 8-9, Eq.
 * "Convolution"), evaluated with a circulant-embedded FFT (algorithm steps
 * 1-7 of Section 2.2).  Conditional simulation (Section 1, Section 4.2) and
 * the adjoint of the implemented map are built on the same machinery.
 *
 * Conventions shared by every entry point:
 *  - Every call is asynchronous on the plan's CUDA stream unless its comment
 *    says otherwise.  Pointers named *_dev are device pointers owned by the
 *    caller; *_host pointers are host memory owned by the caller.  The plan
 *    owns all of its scratch space.  It is allocated by rk_plan_create,
 *    rk_set_sites and rk_set_coef/rk_solve_coef; rk_predict and
 *    rk_predict_group never allocate; rk_simulate and rk_predict_backward
 *    allocate their own scratch on their first call and again whenever the
 *    number of fields (times realisations) grows beyond what they hold.
 *  - Statuses are returned, never raised: no entry point exits, traps or
 *    prints.  After any status other than RK_OK and RK_ERR_CUDA the plan is
 *    still usable; after RK_ERR_CUDA it must be destroyed.
 *  - Grid: nx x ny nodes on extent = {x0, x1, y0, y1} with both end points,
 *    hx = (x1 - x0) / (nx - 1), hy likewise; outputs are row-major
 *    [field][iy][ix] (ix fastest).
 *  - Covariance (Eq. Matern1, Section 3): k(s, s') = sigma2 * phi(|s - s'| /
 *    range), phi(d) = d^nu K_nu(d) / (2^(nu - 1) Gamma(nu)).  nu = 0.5, 1.5,
 *    2.5 use the closed forms; any other 0.2 <= nu <= 8 a table of K_nu
 *    built once per nu (see rk_matern_eval).
 *  - Precision RK_FP64: every step in double.  RK_FP32: scatter and FFT
 *    butterflies in float; the weights, the Cholesky factors and the circulant
 *    eigenvalues in double; the lowest spatial frequencies of F(c*) (where the
 *    Matern spectrum exceeds 1e-2 of its peak) are computed from the sites'
 *    weights in double-float arithmetic (pairs of floats, about 48
 *    significant bits) and replace the float values before the spectrum is
 *    applied.
 */
#ifndef RK_H
#define RK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rk_plan rk_plan;

typedef enum {
  RK_OK = 0,
  RK_ERR_INVALID_ARG = 1,  /* a size, pointer or parameter outside its range  */
  RK_ERR_OBS_OUTSIDE = 2,  /* a site lies outside the extent (or is NaN)      */
  RK_ERR_NOT_PD = 3,       /* a Cholesky factorisation met a non-positive pivot */
  RK_ERR_CE_NEGATIVE = 4,  /* no non-negative circulant embedding found       */
  RK_ERR_CUDA = 5,         /* a CUDA runtime call failed                      */
  RK_ERR_OOM = 6,          /* device allocation failed                        */
  RK_ERR_TIMEOUT = 7,      /* reserved: a bounded device wait gave up         */
  RK_ERR_STATE = 8         /* a call came before the state it needs was set   */
} rk_status;

enum { RK_FP32 = 0, RK_FP64 = 1 };

/* Sizes chosen by a plan (read-only report, see rk_plan_get_info). */
typedef struct {
  int nx, ny, L, M;        /* grid, neighbourhood order, M = (2L)^2            */
  int p1x, p1y;            /* padded grid, P1 = n + 2 (L - 1)                  */
  int px, py;              /* torus size per dimension (2^a 3^b >= 2(n+L-2))   */
  int hx_spec;             /* half-spectrum width px / 2 + 1                   */
  int blk_kx, blk_ky;      /* exact low-frequency block: kx <= blk_kx, |ky| <= blk_ky (FP32 only) */
  int n, B;                /* current sites and fields (0 before they are set) */
  int precision;
  int qx, qy;              /* circulant-embedding torus of rk_simulate (0 until first use) */
} rk_plan_info;

/*
 * rk_plan_create -- algorithm steps 1-2 of Section 2.2 for one covariance.
 * Factors K_N (the M x M covariance among a site's 2L x 2L grid neighbours,
 * shared by all sites because k is stationary and the neighbour order is
 * fixed) and computes the eigenvalues lambda of the circulant embedding of
 * the grid covariance (step 2; embedding per the remark on 2-3-smooth sizes)
 * on the device in double.
 *   out        receives the plan; *out is NULL on failure.
 *   nx, ny     grid nodes per dimension, >= 2.
 *   extent     {x0, x1, y0, y1}, host pointer, x0 < x1, y0 < y1.
 *   nu         Matern smoothness, 0.2 <= nu <= 8 (0.5, 1.5, 2.5: closed forms;
 *              others tabulated, see rk_matern_eval).
 *   range      Matern range (> 0); sigma2 > 0; tau2 >= 0 (nugget).
 *   L          neighbourhood order >= 1, M = (2L)^2 <= 64.
 *   precision  RK_FP32 or RK_FP64.
 *   stream     cudaStream_t to run on (NULL = legacy default stream).
 * Synchronises with the stream before returning.
 */
rk_status rk_plan_create(rk_plan** out, int nx, int ny, const double extent[4],
                         double nu, double range, double sigma2, double tau2,
                         int L, int precision, void* stream);

/* Frees every device buffer of the plan.  NULL is accepted. */
rk_status rk_plan_destroy(rk_plan* plan);

/* Re-targets the plan to another stream. */
rk_status rk_set_stream(rk_plan* plan, void* stream);

/* Copies the plan's sizes into *info (host). */
rk_status rk_plan_get_info(const rk_plan* plan, rk_plan_info* info);

/*
 * rk_set_sites -- algorithm steps 3-4 of Section 2.2 and Eq. (weights).
 * For each site: central box (ix, iy) = clamp(floor((s - x0) / h), 0, n - 2)
 * and local offsets; k_i (covariance with the 2L x 2L neighbours, order
 * q = a + 2L b, a fastest); A_i = K_N^{-1} k_i through the Cholesky factor.
 * For RK_FP32 plans it also forms each site's Fourier factors for the exact
 * low-frequency block.  Resets any coefficients set before.
 *   n        number of sites, >= 1.
 *   xy_dev   device, n x 2 doubles (x, y) row-major.
 * Returns RK_ERR_OBS_OUTSIDE if a site is outside the extent or NaN.
 * Synchronises with the stream (to read the outside-extent flag).
 */
rk_status rk_set_sites(rk_plan* plan, int n, const double* xy_dev);

/*
 * rk_set_sites_async -- rk_set_sites without synchronising: the extent check
 * is latched in the plan's device status word instead of being returned.
 * Sites outside the extent (or NaN) get zero weights.  rk_check_sites reports
 * the latched result.  Lets a caller issue set-up and prediction for many
 * plans on several streams without host round trips.  Sizes must not exceed
 * those of an earlier rk_set_sites on this plan (else RK_ERR_STATE, because
 * growing the plan's buffers would allocate and synchronise).
 */
rk_status rk_set_sites_async(rk_plan* plan, int n, const double* xy_dev);

/*
 * rk_set_sites_group -- rk_set_sites_async for nplans plans at once (1 <=
 * nplans <= 16): the weights of steps 3-4 (Section 2.2) in one launch per
 * neighbourhood size L over all the plans' sites, and the FP32 plans' block
 * factors in one launch, so that the plans of a sweep (Section 3) fill the
 * GPU together.
 *   plans   host array of distinct plans
 *   n       host array, n[k] sites for plans[k] (at most what earlier
 *           rk_set_sites calls sized: no allocation here)
 *   xy      host array of device pointers, xy[k] n[k] x 2 doubles
 * Issued on plans[0]'s stream (block factors on its side stream); no host
 * synchronisation: sites outside the extent are latched per plan and
 * reported by that plan's rk_check_sites once plans[0]'s stream has passed
 * this call (rk_check_sites synchronises only its own plan's stream).
 * Plans must not be in use on other streams meanwhile.  RK_ERR_INVALID_ARG for null or
 * repeated plans, RK_ERR_STATE when n[k] exceeds a plan's sized capacity.
 */
rk_status rk_set_sites_group(rk_plan* const* plans, int nplans, const int* n,
                             const double* const* xy);

/*
 * rk_check_sites -- synchronises with the plan's stream and returns
 * RK_ERR_OBS_OUTSIDE if any site given to rk_set_sites_async since the last
 * check lay outside the extent, RK_OK otherwise; clears the latch.
 */
rk_status rk_check_sites(rk_plan* plan);

/*
 * rk_set_weights -- sets the sparse matrix A of Eq. (6) directly instead of
 * computing it (e.g. weights from another interpolation rule, or the
 * non-stationary variant discussed in Section 6 where k_i comes from a
 * different covariance).  box_dev: device, n x 2 int32 central-box indices
 * (ix in [0, nx - 2], iy in [0, ny - 2]); w_dev: device, n x M doubles in the
 * neighbour order q = a + 2L b.  Resets coefficients; the per-site standard
 * deviations used by rk_simulate are set to zero.  Returns RK_ERR_INVALID_ARG
 * for an index out of range (synchronises to check).
 */
rk_status rk_set_weights(rk_plan* plan, int n, const int* box_dev, const double* w_dev);

/*
 * rk_set_coef -- sets the Kriging coefficients c (Eq. 3) directly, for B
 * fields: c_dev is device, B x n doubles row-major.  Copied into the plan.
 */
rk_status rk_set_coef(rk_plan* plan, int B, const double* c_dev);

/*
 * rk_set_coef_group -- rk_set_coef for nplans plans at once (1 <= nplans <=
 * 16, distinct, each with sites set): one copy launch for all of them, on
 * plans[0]'s stream.  B[k], c_dev[k]: plans[k]'s field count and device
 * coefficients (B[k] x n doubles, n its site count).  Buffers grow on first
 * use (an allocation, so size them before any stream capture).
 * RK_ERR_INVALID_ARG for null, repeated or out-of-range arguments,
 * RK_ERR_STATE for a plan without sites.
 */
rk_status rk_set_coef_group(rk_plan* const* plans, int nplans, const int* B,
                            const double* const* c_dev);

/*
 * rk_solve_coef -- Eq. (3) without covariates: c = M^{-1} z for B fields,
 * M = K_xx + tau2 I (Section 2), by a double-precision Cholesky factorisation
 * of M on the device and two triangular solves.  The factor is kept for
 * rk_simulate and rk_predict_backward.  z_dev: device, B x n doubles (data
 * with any fixed effects X beta already removed).  Returns RK_ERR_NOT_PD if M
 * is not positive definite.  Synchronises with the stream.
 */
rk_status rk_solve_coef(rk_plan* plan, int B, const double* z_dev);

/* rk_set_obs = rk_set_sites followed by rk_solve_coef. */
rk_status rk_set_obs(rk_plan* plan, int n, const double* xy_dev, const double* z_dev, int B);

/*
 * rk_predict -- algorithm steps 5-7 of Section 2.2 (Eqs. 8-9): c* = A^T c on
 * the padded grid, zero-embedded on the px x py torus, convolved with the
 * Matern filter by FFT, and cropped to the nx x ny window (offset L - 1).
 *   out_dev  device, B x ny x nx, float for RK_FP32 plans, double for RK_FP64.
 * Needs rk_set_sites and coefficients (else RK_ERR_STATE).
 */
rk_status rk_predict(rk_plan* plan, void* out_dev);

/*
 * rk_predict_group -- rk_predict for nplans plans at once (1 <= nplans <= 16):
 * the same steps 5-7 of Section 2.2, each pass issued as one launch over the
 * fields of every plan, so that many small predictions (the paper's sweeps
 * over nu and L, Section 3) fill the GPU together.
 *   plans    host array of distinct plans, each with sites and coefficients;
 *            all of one precision and one torus (px, py), which grids of one
 *            size and L within a 2^a 3^b step share.
 *   outs     host array of device pointers, outs[k] as rk_predict's out_dev
 *            for plans[k].
 * Work is issued on plans[0]'s stream (its side stream and events for the
 * FP32 exact block).  Plans must not be in use on other streams meanwhile.
 * RK_ERR_INVALID_ARG for a null or repeated plan, mixed precision or torus;
 * RK_ERR_STATE as rk_predict.  A torus without a compile-time-specialised
 * FFT length is predicted plan after plan on the same stream.
 */
rk_status rk_predict_group(rk_plan* const* plans, int nplans, void* const* outs);

/*
 * rk_predict_static -- rk_predict without any device allocation.  (Not from
 * the paper: it has no counterpart there.)  Some callers cannot allocate
 * device memory at the moment they predict: a process whose device memory is
 * already fully reserved by another allocator, or a latency-critical loop
 * that cannot afford cudaMalloc's implicit device synchronisation.  This
 * entry point computes exactly what rk_predict computes, but keeps the
 * per-call scratch (c*, the two transposed half spectra and the
 * low-frequency block) in one file-scope device array of 32 MiB (33554432
 * bytes) that the library holds on every GPU that loads it, until the
 * process exits.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.
 *   out_dev  device, B x ny x nx in plan precision, as for rk_predict.
 * Returns RK_ERR_INVALID_ARG when the plan's fields need more scratch than
 * the array holds (about 22 MB per field for a 1024 x 1024 grid with L = 3,
 * 5 MB per field at 512 x 512), RK_ERR_STATE before rk_set_sites and
 * coefficients.  The first call on a device looks the array's address up
 * with that device current (cudaGetSymbolAddress); make that first call
 * before any stream capture.  Every call shares the one array and the array
 * keeps the last call's contents, so calls that overlap on the GPU (on
 * different streams or host threads) race and must be serialised by the
 * caller.  Nothing carries over from one call to the next: with fewer than
 * 4096 sites the scatter clears c* in the array before it accumulates into
 * it, and with 4096 or more the tiled scatter writes every element of c*;
 * every other buffer in the array is fully written before it is read.
 */
rk_status rk_predict_static(rk_plan* plan, void* out_dev);

/*
 * rk_predict_host -- the same prediction called with host buffers: copies
 * xy_host (n x 2 doubles) and c_host (B x n doubles) to the device, updates
 * the sites and coefficients, predicts, and copies the B x ny x nx result
 * back into out_host (float or double per the plan precision).  One
 * synchronisation with the stream, at the end; host buffers may be pageable,
 * pinned ones let the copies overlap.  RK_ERR_OBS_OUTSIDE (after the copies)
 * when a site lies outside the extent: that site then carried no weight.
 */
rk_status rk_predict_host(rk_plan* plan, int n, const double* xy_host, int B,
                          const double* c_host, void* out_host);

/*
 * rk_predict_host_group -- rk_predict_host for nplans plans at once (1 <=
 * nplans <= 16, distinct, one precision, one torus): the copies in, the
 * grouped site update (rk_set_sites_group), the coefficients, the grouped
 * prediction (rk_predict_group) and the copies out, issued on plans[0]'s
 * stream with one synchronisation at the end.  When every host buffer is
 * page-locked, the call's stream work is also captured as a CUDA graph (held
 * by plans[0]) and later calls with the same plans, sizes and pointers replay
 * it, as long as no plan buffer has been allocated or released meanwhile.
 *   n[k], xy_host[k]   sites of plans[k] (host, n[k] x 2 doubles)
 *   B[k], c_host[k]    its coefficients (host, B[k] x n[k] doubles)
 *   out_host[k]        its result (host, B[k] x ny x nx, plan precision)
 * Device buffers grow on first use.  RK_ERR_OBS_OUTSIDE when any plan saw a
 * site outside its extent (its latch is cleared); the other errors as for
 * rk_set_sites_group and rk_predict_group.
 */
rk_status rk_predict_host_group(rk_plan* const* plans, int nplans, const int* n,
                                const double* const* xy_host, const int* B,
                                const double* const* c_host, void* const* out_host);

/*
 * rk_simulate -- conditional simulation (Section 1: unconditional draw, then
 * Kriging of the simulated data; Section 6: circulant embedding).  For each
 * of the B data fields z given to rk_solve_coef and each realisation
 * t < R: an unconditional field f_u on the padded grid from a circulant
 * embedding (torus 2^a 3^b >= 2 (P1 - 1), grown until its eigenvalues are
 * non-negative), site values z_u = A_i f_u[N(i)] + s_i xi + tau eps with
 * s_i^2 = max(0, sigma2 - k_i^T A_i), coefficients c = M^{-1} (z - z_u), and
 * f_c = rapid prediction of c + f_u on the window.  Noise is Philox4x64-10
 * keyed by (seed, 0): one call per four consecutive indices (counter
 * (index >> 2, realisation or pair, stream, 0), index j taking word j mod 4),
 * Box-Muller on a word's high and low 32-bit halves, u(x) = (x + 1/2) 2^-32.
 * Stream 1 is the embedding's noise at torus index kx * qy + ky for the
 * realisation pair, stream 2 the site noise at site i for the realisation.
 *   out_dev  device, B x R x ny x nx in plan precision.
 * Needs rk_solve_coef (else RK_ERR_STATE); RK_ERR_CE_NEGATIVE if no
 * embedding up to four-fold growth is non-negative.
 */
rk_status rk_simulate(rk_plan* plan, int R, unsigned long long seed, void* out_dev);

/*
 * rk_predict_backward -- adjoint of the implemented map
 * (z, log range, log sigma2) -> g_hat (the paper has no gradient).
 * Given gbar = d loss / d g_hat (device, B x ny x nx, plan precision):
 *   grad_z_dev          device, B x n doubles, d loss / d z;
 *   grad_log_range_dev  device, B doubles;
 *   grad_log_sigma2_dev device, B doubles.
 * Any of the three outputs may be NULL to skip it.  Needs rk_solve_coef.
 */
rk_status rk_predict_backward(rk_plan* plan, const void* gbar_dev, double* grad_z_dev,
                              double* grad_log_range_dev, double* grad_log_sigma2_dev);

/*
 * rk_debug_copy -- copies an internal buffer into a caller device buffer for
 * testing (dst_dev must hold the stated bytes).  what: 0 = box indices
 * (n x 2 int32: ix, iy), 1 = weights (n x M doubles), 2 = spectrum lambda
 * (px/2+1 columns x py, plan precision, scaled by 1/(px py)),
 * 3 = c* of field 0 (p1y x p1x, plan precision), 4 = coefficients c
 * (B x n doubles).  Synchronises.
 */
rk_status rk_debug_copy(rk_plan* plan, int what, void* dst_dev, size_t bytes);

/*
 * Per-kernel timing for measurement (not part of the method).  While enabled,
 * every kernel launched by rk_predict / rk_simulate / rk_predict_backward is
 * bracketed by CUDA events on the plan's stream, and its algorithmic bytes
 * (the bytes its inputs and outputs occupy, as stated in the library's design
 * notes) are recorded.  rk_profile_read synchronises the recorded events and
 * fills up to max entries (one per kernel name) with launches, total
 * milliseconds, total algorithmic bytes and, for passes bound by arithmetic
 * at FP64 precision (on the FP64 pipe, or in double-float on the FP32 pipe:
 * the pipe field), total algorithmic operations (adds and multiplies, a fused
 * multiply-add counting two); it returns the number of entries.
 */
typedef struct {
  char name[32];
  int launches;
  double total_ms;
  double bytes;
  double flops;   /* algorithmic FP64-precision operations of arithmetic-bound passes, else 0 */
  int pipe;       /* 0: memory-bound pass; 64: FP64 pipe; 2: double-float on the FP32 pipe */
} rk_profile_entry;
rk_status rk_profile_enable(int on);
int rk_profile_read(rk_profile_entry* out, int max);

/*
 * rk_solve_gls -- universal Kriging, Eqs. (2)-(3) of Section 2: with site
 * covariates X, the generalised least squares estimate
 * beta = (X^T M^-1 X)^-1 X^T M^-1 z and the coefficients
 * c = M^-1 (z - X beta) of the spatial part (the plan's coefficients, as
 * rk_solve_coef sets them); the plan keeps z - X beta as its data (the
 * conditional simulation conditions on it).  M^-1 X and M^-1 z take one pass
 * of the plan's FP64 Cholesky solves (double-float updates for RK_FP32).
 *   B       fields, >= 1; z_dev device, B x n doubles.
 *   q       covariates, 1 <= q <= 16 and q < n; X_dev device, n x q doubles
 *           (row i: the covariates of site i).
 *   beta_dev  device, B x q doubles: the estimates.
 * Allocates its scratch ((q + B) n + q (q + B) doubles) on first use and when
 * it grows.  RK_ERR_NOT_PD when M or X^T M^-1 X is not positive definite.
 * Synchronises with the stream.
 */
rk_status rk_solve_gls(rk_plan* plan, int B, const double* z_dev, int q, const double* X_dev,
                       double* beta_dev);

/*
 * rk_add_trend -- Eq. (5): f = X_g beta + g_hat, the fixed effects added in
 * place to a predicted grid.
 *   Xg_dev    device, q x ny x nx doubles (covariate a at every node).
 *   beta_dev  device, B x q doubles (e.g. from rk_solve_gls).
 *   out_dev   device, B x ny x nx in plan precision (rk_predict's output).
 */
rk_status rk_add_trend(rk_plan* plan, int B, int q, const double* Xg_dev, const double* beta_dev,
                       void* out_dev);

/*
 * rk_simulate_group -- rk_simulate for several plans in one call: R
 * realisations of every data field of every plan (plan k's output as
 * rk_simulate's, B_k x R x ny_k x nx_k), the noise of each plan exactly as
 * rk_simulate draws it (same seed: the same realisations).  Plans that share
 * their sites, covariance and precision (e.g. one data set predicted at
 * several grid resolutions) share M = K_xx + tau^2 I, and all their
 * right-hand sides go through one pass of the triangular solves with the
 * first plan's factor (the dominant cost of a simulation); up to 2048
 * realisations in total, otherwise plan after plan.  Runs on the first plan's
 * stream; allocates scratch as rk_simulate does and, for the shared solve,
 * (sum of B_k R) x n doubles in the first plan.
 *   nplans  1 .. 16 distinct plans;  outs  device pointers, one per plan.
 * RK_ERR_STATE / RK_ERR_CE_NEGATIVE as rk_simulate; synchronises once to
 * compare the plans' sites.
 */
rk_status rk_simulate_group(rk_plan* const* plans, int nplans, int R, unsigned long long seed,
                            void* const* outs);

/*
 * rk_exact_predict -- exact Kriging, Eq. (4) of Section 2, at np points:
 * g_hat(s_p) = sum_i k(s_p, s_i) c_i with the plan's sites and coefficients
 * (c = M^-1 z from rk_solve_coef), summed in double over all n sites.  For
 * checking the rapid predictor against exact Kriging (the paper's factorial
 * study, Section 3.1) at a few points; O(np n).
 *   pts_dev  device, np x 2 doubles;  out_dev  device, B x np doubles.
 * RK_ERR_STATE before sites (not weights) and coefficients; B <= 16.
 */
rk_status rk_exact_predict(rk_plan* plan, int np, const double* pts_dev, double* out_dev);

/*
 * rk_draw_obs -- observations drawn from the model at the plan's sites:
 * z = L_M xi with L_M the lower Cholesky factor of M = K_xx + tau^2 I (formed
 * here when the sites have none yet), so that z ~ N(0, M) for standard
 * normal xi: the simulated data of Section 3.1's study.
 *   xi_dev, z_dev  device, B x n doubles.
 */
rk_status rk_draw_obs(rk_plan* plan, int B, const double* xi_dev, double* z_dev);

/*
 * rk_kernel_error -- Lambda(Omega, s*) of Section 3.2: the largest error of
 * the local kernel approximation, sup over s in Omega of
 * |k_approx(s, s*) - k(s, s*)|, k_approx(s, s*) = sum_q W_q k(s, s_q) over the
 * 2L x 2L neighbours of s* with K_N W = k(s*) (Eq. weights; Cholesky in
 * double), for s* at the centre of the central box (node indices
 * ((nx - 2) / 2, (ny - 2) / 2)).  Omega is the plan's extent; the supremum is
 * taken on the mesh of spacing (hx / sub, hy / sub) covering it (its nodes
 * include the grid's).  Uses the plan's covariance (sigma2 scales Lambda).
 *   sub   1 .. 64 mesh points per grid spacing;  out  host, one double.
 * Needs nx, ny >= 2L.  RK_ERR_NOT_PD when K_N's factorisation fails.
 * Allocates 65 doubles on first use; synchronises with the stream.
 */
rk_status rk_kernel_error(rk_plan* plan, int sub, double* out);

/*
 * rk_interp -- prediction at irregular locations from a predicted grid, the
 * extension proposed in Section 6 (Conclusion & Discussion): predict onto a
 * fine regular mesh with the rapid method, then interpolate off the mesh by
 * a local polynomial rule.  The rule here is tensor-product Lagrange
 * interpolation with K points per axis (K = 2: bilinear; 4: cubic; 6:
 * quintic): for a target with grid coordinate gx = (x - x0) / hx the stencil
 * is the K nodes from clamp(floor(gx) - K/2 + 1, 0, nx - K), likewise in y;
 * weights and sums in double.
 *   grid_dev  device, B x ny x nx in plan precision (e.g. rk_predict's output).
 *   B         fields, >= 1.
 *   np        targets, >= 0; xy_dev device, np x 2 doubles (x, y).
 *   K         2, 4 or 6 (at most nx and ny).
 *   out_dev   device, B x np in plan precision.
 * Returns RK_ERR_OBS_OUTSIDE when a target lies outside the extent (its
 * outputs are NaN, the others are valid); RK_ERR_INVALID_ARG for bad sizes.
 * Synchronises with the stream (to read the outside-extent flag).
 */
rk_status rk_interp(rk_plan* plan, const void* grid_dev, int B, int np, const double* xy_dev,
                    int K, void* out_dev);

/*
 * rk_matern_eval -- the library's Matern correlation for a smoothness without
 * a closed form, evaluated on the host (no GPU).  Plans with nu other than
 * 1/2, 3/2, 5/2 (0.2 <= nu <= 8, at most 8 distinct values per process) use
 * phi(t) = 2^(1-nu) / Gamma(nu) t^nu K_nu(t) (Eq. Matern1) and its log-range
 * derivative -t phi'(t) = 2^(1-nu) / Gamma(nu) t^(nu+1) K_(nu-1)(t) from a
 * table built once per nu: K_nu by the trapezoidal rule on its integral
 * representation in long double, then Chebyshev series of degree 20 on
 * segments [2^-(k+1), 2^-k] (k < 60) and [1 + j, 2 + j] up to the tail where
 * both fall below 1e-20 (zero beyond; for 0 < t < 2^-60 the value at 2^-60).
 * The device kernels evaluate the same table.
 *   which  0: phi(t); 1: -t phi'(t).   t, out: host arrays of n doubles.
 * RK_ERR_INVALID_ARG for nu outside [0.2, 8] or bad arguments.
 */
rk_status rk_matern_eval(double nu, int which, int n, const double* t, double* out);

/*
 * FFT pass variants and their tuner (no counterpart in the paper: how the
 * transforms of steps 6-7 are run).  Each of the three passes of a
 * compile-time torus length n (rows of c* forward, columns forward-spectrum-
 * inverse, rows inverse; pass 0, 1, 2) has variant 0, one transform per
 * radix stage in shared memory, and variants 1.., register-resident
 * transforms with E elements per thread (radix plan) and V transforms per
 * CTA.  The first plan created with a torus length (per precision, per
 * process) times every variant of each pass on a synthetic batch and keeps
 * the fastest; RK_FFT_TUNE=0 in the environment keeps variant 1 instead.
 * With RK_FFT_CACHE=path the choices are read from that text file (lines
 * "n precision pass variant") when it has them for the length, and a process
 * that tunes appends its choices there (so that, e.g., a profiled run takes
 * the choices of the plain run before it).
 * The choice is process-wide; the per-length twiddle tables are per device.
 *
 * rk_fft_variants     number of variants of a pass (1 for lengths with no
 *                     specialisation, which run the generic kernels).
 * rk_fft_get_choice   *cand = the variant in use, -1 before the first plan.
 * rk_fft_set_choice   forces a variant (RK_ERR_INVALID_ARG out of range);
 *                     uploads its tables to the current device.
 * rk_fft_variant_info *e, *v of a variant (0, 0 for variant 0).
 * rk_fft_tune         re-times every variant of the three passes on stream
 *                     (NULL: legacy default) and keeps the fastest; when
 *                     times_ms is not NULL it receives 24 doubles,
 *                     times_ms[pass * 8 + variant] = mean milliseconds per
 *                     launch (-1 where a variant could not launch).
 *                     Allocates and frees its test buffers; synchronises.
 */
int rk_fft_variants(int n, int precision, int pass);
rk_status rk_fft_get_choice(int n, int precision, int pass, int* cand);
rk_status rk_fft_set_choice(int n, int precision, int pass, int cand);
rk_status rk_fft_variant_info(int n, int precision, int pass, int cand, int* e, int* v);
rk_status rk_fft_tune(int n, int precision, void* stream, double* times_ms);

/* A static string naming the status. */
const char* rk_status_string(rk_status s);

#ifdef __cplusplus
}
#endif

#endif /* RK_H */
