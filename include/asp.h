/*
 * libasp -- the Asp-Clean2016 minor cycle on one GB300 GPU (sm_103a).
 *
 * Zhang, Bhatnagar, Rau & Zhang (2016), "Efficient implementation of the
 * adaptive scale pixel decomposition algorithm".  The PSF is approximated by a
 * single Gaussian (alpha_b, omega_b) (Sect. 3), so each candidate component is
 * fitted as a PSF-convolved Gaussian directly to the residual image (Eq. 6) by
 * Levenberg-Marquardt, then deconvolved analytically (Eqs. 7-8); the residual
 * is updated with the full PSF (Sect. 2 step 3) and initial values come from a
 * peak search, simple or multi-scale smoothed (Sect. 2 step 1, Sect. 3).
 *
 * Conventions for every call:
 *  - Images are FP32, row-major, y the slow axis; pixel centres sit at integer
 *    coordinates (x = column, y = row); flat index = y * W + x.
 *  - The PSF is a 2H x 2W FP32 array whose zero lag is at [H, W] (so
 *    B[p - q + (H, W)] exists for every pair of image pixels p, q).
 *  - "_dev" pointers are device pointers of the current CUDA device; "_host"
 *    pointers are host memory (pageable or pinned).  The library copies what
 *    it is given: it never keeps a caller pointer after a call returns.
 *  - Every call enqueues its work on the context's stream; calls that return
 *    values synchronise that stream before returning.
 *  - Errors are returned, never thrown; nothing aborts.  After ASP_ERR_CUDA or
 *    ASP_ERR_TIMEOUT the context answers ASP_ERR_STATE to everything except
 *    asp_destroy and the getters of the last error.
 *  - A context is not thread-safe: one host thread at a time.
 */
#ifndef ASP_H
#define ASP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct asp_ctx asp_ctx;

typedef enum {
    ASP_OK = 0,
    ASP_ERR_INVALID_ARG = 1,   /* bad pointer, size or parameter */
    ASP_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    ASP_ERR_OOM = 3,           /* device allocation failed */
    ASP_ERR_NAN = 4,           /* non-finite input or result */
    ASP_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
    ASP_ERR_NOT_CONVERGED = 6, /* reserved: fits report status in asp_fit_info */
    ASP_ERR_STATE = 7,         /* context unusable after an earlier failure */
    ASP_ERR_UNSUPPORTED = 8,   /* size beyond a compiled-in limit */
    ASP_ERR_CAPACITY = 9       /* component list full */
} asp_status;

/* Initial-value modes (Sect. 3): AUTO applies the 5 % area switch. */
typedef enum { ASP_INIT_AUTO = 0, ASP_INIT_SIMPLE = 1, ASP_INIT_SMOOTH = 2 } asp_init_mode;
/* Peak-search modes for asp_find_peak. */
typedef enum { ASP_PEAK_SIMPLE = 0, ASP_PEAK_SMOOTH = 1 } asp_peak_mode;
/* Residual update form.  DIRECT: separable passes over the PSF rows and
 * columns the terms need (cost ~ sum over terms of taps x image pixels).
 * FFT: the iteration's change image dC convolved with B as one product on
 * the zero-padded 2H x 2W grid (cuFFT, FP32; cost independent of the number
 * and widths of the terms).  AUTO: FFT for images of at least
 * ASP_SUB_FFT_MIN_PIXELS pixels, DIRECT below. */
typedef enum { ASP_SUB_AUTO = 0, ASP_SUB_DIRECT = 1, ASP_SUB_FFT = 2 } asp_sub_mode;
#define ASP_SUB_FFT_MIN_PIXELS 262144   /* 512 x 512 */
/* Levenberg-Marquardt termination codes (asp_fit_info.status). */
typedef enum { ASP_LM_CONVERGED = 0, ASP_LM_CAP = 1, ASP_LM_STALLED = 2 } asp_lm_status;
/* Why a minor cycle stopped (asp_cycle_stats.stop_reason). */
typedef enum {
    ASP_STOP_NONE = 0, ASP_STOP_ITER = 1, ASP_STOP_NOISE = 2, ASP_STOP_CAPACITY = 3
} asp_stop_reason;

/* Largest active set one fit accepts (members fitted jointly). */
#define ASP_KMAX 50

/* A PSF-convolved Gaussian a exp(-((x-x0)^2+(y-y0)^2)/(2 w^2)): the fitted
 * function of Eq. 6, (alpha_ic, x_ic, y_ic, omega_ic). */
typedef struct { double amp, x, y, width; } asp_gauss;

/* A deconvolved model component (Eqs. 7-8): flux F = 2 pi alpha omega^2 (for a
 * point: F itself), amplitude alpha, centre, width omega (0 for a point). */
typedef struct {
    double flux, amp, x, y, width;
    int32_t is_point;
    int32_t reserved;
} asp_component;

/* Elliptical variant (the paper's circular Gaussians of Sect. 3 with a 2 x 2
 * shape): a exp(-(A dx^2 + 2 B dx dy + C dy^2) / 2), (dx, dy) the offset
 * from (x, y) and P = [[A, B], [B, C]] (pxx, pxy, pyy) the precision matrix,
 * i.e. the inverse covariance.  For a circle of width w: A = C = 1 / w^2,
 * B = 0. */
typedef struct { double amp, x, y, pxx, pxy, pyy; } asp_gauss_ell;

/* A deconvolved elliptical component: covariances add under convolution,
 * so Sigma_i = Sigma_ic - Sigma_beam (Eq. 7's analogue), and flux is
 * conserved (Eq. 8's analogue): flux F = a_ic sqrt(det Sigma_ic) / (alpha_b
 * sqrt(det Sigma_b)), amp = F / (2 pi sqrt(det Sigma_i)); (sxx, sxy, syy)
 * the covariance Sigma_i.  A point (Sigma_i = 0, amp = F) when the smaller
 * eigenvalue of Sigma_ic - Sigma_b is at most 1e-3 times the smaller
 * eigenvalue of Sigma_b (for a circular beam exactly the circular rule). */
typedef struct {
    double flux, amp, x, y, sxx, sxy, syy;
    int32_t is_point;
    int32_t reserved;
} asp_component_ell;

/* Largest elliptical active set (6 parameters a member). */
#define ASP_ELL_KMAX 33

/* Peak-search result.  SIMPLE: the largest |R| (lowest index on ties), init
 * (R(p*), x*, y*, omega_b).  SMOOTH: the largest |S_j| over scales and pixels
 * (ties: lower scale, then lower index); init (S/(sqrt(pi) s), x*, y*,
 * max(s, omega_b)). */
typedef struct {
    int64_t index;
    int32_t x, y;
    float value;          /* R(p*) or S_j*(p*) */
    float scale;          /* s_j* (SMOOTH) or 0 */
    int32_t mode;         /* asp_peak_mode */
    int32_t scale_index;  /* j* or -1 */
    double a0, x0, y0, w0;
} asp_peak;

/* Outcome of one Levenberg-Marquardt fit. */
typedef struct {
    int32_t iters;        /* damped solves (accepted or rejected) */
    int32_t passes;       /* pixel passes over the window (1 + valid trials) */
    int32_t status;       /* asp_lm_status */
    int32_t k;            /* members fitted */
    int32_t x0, x1, y0, y1; /* fit window (inclusive) */
    double chi2_init, chi2_final, lambda;
    int64_t pixel_evals;  /* passes x window pixels */
} asp_fit_info;

/* Minor-cycle parameters.  Defaults from asp_default_params. */
typedef struct {
    float gain;           /* loop gain for a new component (Sect. 4: 0.35) */
    int32_t k_max;        /* active-set cap (1..ASP_KMAX) */
    int32_t lm_max_iter;  /* damped solves per fit (50) */
    double lm_lambda0;    /* 1e-3 */
    double lm_rtol;       /* predicted / actual relative chi2 decrease (1e-7) */
    double lm_xtol;       /* relative step size (1e-7) */
    float noise_sigma;    /* <= 0: 1.4826 x MAD of the dirty image */
    float stop_ksigma;    /* stop when max|R| < stop_ksigma * noise_sigma (3) */
    int32_t n_scales;     /* smoothing scales omega_b 2^j, j < n_scales (6) */
    float area_frac;      /* simple-method switch threshold (Sect. 3: 0.05) */
    int32_t init_mode;    /* asp_init_mode */
    double tau;           /* active-set retention threshold (1e-3) */
    int32_t retained_cap; /* retained-list cap (0: 8 x k_max) */
    int32_t max_components; /* component-list capacity (0: 65536) */
    int32_t fit_px_per_cta; /* launch shape of the LM fit: window pixels per CTA
                               (0: 96; clamped to [32, 12288]); changes the
                               grid and so the FP32 summation order, not the
                               method */
    int32_t major_every;    /* 0: every iteration subtracts with the full PSF
                               (Sect. 2 step 3).  n > 0: minor/major split in
                               the manner of Clark CLEAN (Sect. 1, Sect. 3):
                               minor iterations subtract each component's
                               single-Gaussian-beam image (Eqs. 7-8 inverted)
                               locally, and after every n of them, and at the
                               end of each asp_minor_cycle call, the residual
                               is recomputed exactly as D - B * M by an FFT
                               convolution.  Contexts only (not batches). */
    int32_t sub_mode;       /* asp_sub_mode: how the per-iteration residual
                               update R -= B * dC (Sect. 2 step 3, full PSF)
                               is computed.  Both forms take the same terms
                               with the same sampled axis weights and point
                               deposits and differ only in rounding.  Unused
                               with major_every > 0.  Batches always take the
                               direct passes (FFT rejected). */
} asp_params;

/* Totals of asp_minor_cycle since asp_init (or the last asp_set_state). */
typedef struct {
    int64_t iterations;   /* minor-cycle iterations done */
    int64_t components;   /* components in the model */
    int64_t pixel_evals;  /* LM pixel evaluations (window pixels x passes) */
    int64_t lm_iters;     /* damped solves */
    int64_t lm_passes;    /* pixel passes */
    double peak_abs;      /* current max |R| */
    int32_t stop_reason;  /* asp_stop_reason of the last call */
    int32_t reserved;
    /* Algorithmic work (the method's own arithmetic, not what the kernels
     * happen to execute): LM pixel passes, 15K + 1 + (4K+1)(4K+2) FP32 flops
     * per pixel evaluation with K members; subtraction as separable passes,
     * 2 nx (H+ny-1) W + 2 ny H W flops per term, bytes = PSF regions read
     * once + residual read and written once; smoothing 4 (2m+1) H W flops
     * per scale and smoothing iteration. */
    double fit_flops, sub_flops, sub_bytes, smooth_flops;
    /* Wall time of the LM fits split into pixel passes, reductions (CTA and
     * cross-CTA, barriers included) and LM logic + damped solves, as seen by
     * the fit kernel's first CTA (%globaltimer). */
    double fit_pass_ms, fit_reduce_ms, fit_solve_ms;
    double fit_factor_ms, fit_subst_ms;   /* parts of fit_solve_ms: damped solves, LM bookkeeping */
    int64_t fit_refinements;  /* FP64 iterative-refinement steps of the FP32-factored solves */
    int64_t fit_fallbacks;    /* solves that fell back to an FP64 factor */
    int64_t learned_fits;     /* fits started from the network's proposal */
    int64_t learned_refits;   /* of those, refitted from the plain start by the fallback rule */
    int64_t learned_kept;     /* of those, whose learned-start result was kept */
    double fit_ex2;           /* exponentials the LM passes evaluate: K per pixel evaluation */
    int64_t smooth_iters;     /* iterations whose initial values came from the smoothing search */
} asp_cycle_stats;

/* One minor-cycle iteration as recorded on the device. */
typedef struct {
    int32_t t, mode, k, status;
    int32_t iters, passes, x0, x1, y0, y1;
    int32_t new_index, n_terms;
    float peak_value, init_scale;
    double chi2_init, chi2_final;
    double a0, x0_init, y0_init, w0;
} asp_iter_record;

const char* asp_status_string(asp_status s);
void asp_default_params(asp_params* p);

/* Create a context: copies dirty (H x W) and psf (2H x 2W) from device
 * memory, fits the single-Gaussian beam (alpha_b, omega_b) to the PSF main
 * lobe (Sect. 3) and finds the first peak.  stream: a cudaStream_t (NULL:
 * the legacy default stream).  On error *out is NULL. */
asp_status asp_init(const asp_params* p, int H, int W, const float* dirty_dev, const float* psf_dev,
                    void* stream, asp_ctx** out);
/* Same as asp_init with host-memory inputs (the copy is part of the call). */
asp_status asp_init_host(const asp_params* p, int H, int W, const float* dirty_host,
                         const float* psf_host, void* stream, asp_ctx** out);
asp_status asp_destroy(asp_ctx* ctx);
/* Last error message of this context ("" if none). */
const char* asp_last_error(const asp_ctx* ctx);

/* Beam (alpha_b, omega_b) and the fitted centre (PSF array coordinates). */
asp_status asp_get_beam(asp_ctx* ctx, double* alpha_b, double* omega_b, double* x_b, double* y_b);

/* Peak search on the current residual (Sect. 2 step 1; Sect. 3 simple
 * method).  mode: asp_peak_mode. */
asp_status asp_find_peak(asp_ctx* ctx, int mode, asp_peak* out);

/* Joint LM fit of n Gaussians (Eq. 6) to the current residual.  The last
 * n_old members are taken as already subtracted: their initial Gaussians are
 * added back to form the target T = R + sum_old g(init).  The window is the
 * bounding box of the members' boxes (half-width max(5, ceil(4 w)) around the
 * rounded centre), clipped to the image.  Writes n fitted Gaussians to out
 * (host) and the fit outcome to info (host).  1 <= n <= k_max. */
asp_status asp_fit_active_set(asp_ctx* ctx, const asp_gauss* init, int n, int n_old,
                              asp_gauss* out, asp_fit_info* info);

/* Normal equations of the Eq. 6 objective at theta over a given window
 * (inclusive bounds, clipped), target T = R + sum of the last n_old members:
 * A = J^T J (4n x 4n, row-major, full), g = J^T r, chi2 = r^T r.  Host
 * outputs.  This is the LM pixel pass on its own. */
asp_status asp_eval_normal_equations(asp_ctx* ctx, const asp_gauss* theta, int n, int n_old,
                                     int x0, int x1, int y0, int y1,
                                     double* A_host, double* g_host, double* chi2_host);

/* Levenberg-Marquardt (Marquardt 1963, the minimiser of Eq. 6) restarted at
 * any point of a fit: the fit of asp_fit_active_set defined by init, n and
 * n_old (window = bounding box of the init members' boxes; target T = R +
 * the last n_old members' init Gaussians; trial bounds), but LM starts at
 * start (n rows, host; NULL: init) with damping lambda = lambda0 (> 0,
 * finite) and stops after max_iter damped solves (>= 0).  Besides the kept
 * point (out) and the outcome (info; info->lambda is the damping after the
 * last decision, info->chi2_init chi^2 at start), it returns the last
 * proposed trial point theta + delta of the last damped solve (trial_out, n
 * rows, host; may be NULL) and chi^2 of the last pixel pass (chi2_trial,
 * host; may be NULL), which is chi^2 at that trial point when it was
 * evaluated (info->passes counts the passes: the start plus each evaluated
 * trial).  With max_iter = 1 this is one Marquardt step from (theta,
 * lambda): one damped solve, the trial pass and the accept decision -- the
 * hook the step-by-step parity tests and measurements use.  Errors as
 * asp_fit_active_set; ASP_ERR_INVALID_ARG for a bad start, lambda0 or
 * max_iter. */
asp_status asp_fit_lm(asp_ctx* ctx, const asp_gauss* init, int n, int n_old, const asp_gauss* start, double lambda0,
                      int max_iter, asp_gauss* out, asp_fit_info* info, asp_gauss* trial_out, double* chi2_trial);

/* Asp-Clean2004's objective (Sect. 2, Eq. 3), the system the paper
 * accelerates: Levenberg-Marquardt on chi^2 = || T - B * sum_k g_k ||^2 over
 * the whole image, g_k the UNCONVOLVED component a exp(-r^2 / 2 w^2) of each
 * member (rows of init: amplitude, centre, width of the component itself),
 * B the full PSF applied by an FFT convolution on the 2H x 2W grid in every
 * evaluation (cuFFT, FP32), T the residual with the last n_old members'
 * init components added back through B.  The LM rules are
 * asp_fit_active_set's (context LM settings; trial widths in (omega_min,
 * max(H, W)], centres inside the image; a trial costs the model's
 * convolution, an accepted point the 4n Jacobian convolutions).  With a
 * Gaussian PSF its optimum maps to Eq. 6's through Eqs. 7-8.  The LM
 * iterations run on the host, the images, FFTs and sums on the device.
 * 1 <= n <= 8 (ASP_ERR_UNSUPPORTED beyond).  The first call allocates its
 * buffers (33 zero-padded images of 2H x 2W, their transforms) and plans,
 * kept until asp_destroy.  info->pixel_evals counts evaluations x H W. */
asp_status asp_fit_2004(asp_ctx* ctx, const asp_gauss* init, int n, int n_old, double omega_min, asp_gauss* out,
                        asp_fit_info* info);

/* Elliptical beam: the circular beam's fit region (the pixels within
 * ceil(3 omega_init) of the PSF's zero lag, omega_init its half-maximum
 * width), Levenberg-Marquardt on the elliptical model started from the
 * circular beam (A = C = 1 / omega_b^2, B = 0); trial principal widths in
 * (0.25 omega_init, region extent].  out: (alpha_b, x_b, y_b, A_b, B_b,
 * C_b) on the 2H x 2W PSF grid (zero lag at (W, H)).  ASP_ERR_NAN if the
 * fit ends without a positive-definite shape.  The minor cycle keeps its
 * circular beam. */
asp_status asp_fit_beam_elliptical(asp_ctx* ctx, asp_gauss_ell* out);

/* Eq. 6 with elliptical members: as asp_fit_active_set (same window rule,
 * from the major width 1 / sqrt(mu_min(P)); same LM rules and launch), the
 * last n_old members of init added back to the residual as the target,
 * trial points positive definite with principal widths in (0.25 omega_b,
 * window extent] and centres in the window.  1 <= n <= ASP_ELL_KMAX
 * (ASP_ERR_UNSUPPORTED beyond); ASP_ERR_INVALID_ARG for a non-finite value
 * or a shape that is not positive definite. */
asp_status asp_fit_elliptical(asp_ctx* ctx, const asp_gauss_ell* init, int n, int n_old, asp_gauss_ell* out,
                              asp_fit_info* info);

/* Eqs. 7-8 for elliptical shapes (see asp_component_ell) on the device, for
 * n fitted (PSF-convolved) Gaussians in against the beam (alpha_b, P_b) in
 * beam (e.g. from asp_fit_beam_elliptical).  n <= ASP_ELL_KMAX;
 * ASP_ERR_INVALID_ARG for a shape that is not positive definite. */
asp_status asp_deconvolve_elliptical(asp_ctx* ctx, const asp_gauss_ell* in, int n, const asp_gauss_ell* beam,
                                     asp_component_ell* out);

/* R -= B * (gain * sum_i c_i) with the full PSF (Sect. 2 step 3); c_i is
 * component i sampled on the grid (a flux-normalised Gaussian on the box
 * |q - centre|_inf <= ceil(5 w) + 1 if w >= 0.5 px and not a point, else a
 * bilinear deposit).  A negative flux adds the component back.  n <= 2 x
 * ASP_KMAX. */
asp_status asp_subtract(asp_ctx* ctx, const asp_component* comps, int n, float gain);

/* R -= gain * sum_i b_i: component i through the PSF's single-Gaussian
 * approximation (alpha_b, omega_b) -- the Gaussian (alpha_b omega_b^2 F_i /
 * omega_ic^2, x_i, y_i, omega_ic), omega_ic^2 = omega_i^2 + omega_b^2
 * (Eqs. 7-8 inverted) -- on the box |q - centre|_inf <= ceil(5 omega_ic) +
 * 1, clipped: the minor cycle's update when asp_params.major_every > 0.
 * Components whose own sampling box lies outside the image are skipped, as
 * in asp_subtract.  n <= 2 x ASP_KMAX.  Finds the next peak. */
asp_status asp_subtract_beam(asp_ctx* ctx, const asp_component* comps, int n, float gain);

/* Run up to n_iter minor-cycle iterations (Sect. 2 steps 1-4 with the
 * Sect. 3 objective, deconvolution and initial-value switch); the loop stops
 * early when max|R| < stop_ksigma * noise_sigma.  Totals to out (may be NULL).
 * With asp_params.major_every = m > 0 a major cycle (the exact residual D -
 * B * M) follows every m iterations of the call and ends the call, so the
 * residual is exact on return. */
asp_status asp_minor_cycle(asp_ctx* ctx, int n_iter, asp_cycle_stats* out);

/* Multi-scale smoothed residual S_j (unit-L2 Gaussian of scale s_j, zero
 * padding) written to out_dev (H x W, device).  scale_index < asp_num_scales. */
asp_status asp_smooth(asp_ctx* ctx, int scale_index, float* out_dev);
asp_status asp_num_scales(asp_ctx* ctx, int* n, double* scales_host /* >= n entries or NULL */);

/* Residual access.  asp_residual_ptr: borrowed device pointer, valid until
 * asp_destroy; writes through it are the caller's responsibility (call
 * asp_refresh_peak afterwards). */
asp_status asp_residual_ptr(asp_ctx* ctx, float** residual_dev);
asp_status asp_copy_residual(asp_ctx* ctx, float* dst, int dst_on_host);
asp_status asp_set_residual(asp_ctx* ctx, const float* src, int src_on_host);
asp_status asp_refresh_peak(asp_ctx* ctx);

/* Model access.  asp_get_components copies min(cap, count) components to
 * host memory and sets *count to the total. */
asp_status asp_get_components(asp_ctx* ctx, asp_component* out_host, int cap, int* count);
asp_status asp_get_history(asp_ctx* ctx, asp_iter_record* out_host, int cap, int* count);
asp_status asp_get_stats(asp_ctx* ctx, asp_cycle_stats* out);

/* Minor-cycle state beyond the residual: the component list, the retained
 * (active) list most recent first, the iteration counter and the last
 * iteration's (omega_i, omega_0) used by the init-mode switch.  All host. */
asp_status asp_get_state(asp_ctx* ctx, asp_component* comps, int comp_cap, int* n_comp,
                         int* retained, int ret_cap, int* n_ret, int64_t* t,
                         double* last_wi, double* last_w0);
asp_status asp_set_state(asp_ctx* ctx, const asp_component* comps, int n_comp,
                         const int* retained, int n_ret, int64_t t, double last_wi,
                         double last_w0);
/* The most recent LM fit of this context (minor-cycle iteration or
 * asp_fit_active_set): the fitted PSF-convolved Gaussians, members in fit
 * order (new member first in a minor cycle), and its outcome.  Copies
 * min(cap, n) rows to host memory and sets *n to the member count. */
asp_status asp_get_last_fit(asp_ctx* ctx, asp_gauss* out_host, int cap, int* n, asp_fit_info* info);

/* Restart on a new dirty image of the same size without reallocating: copies
 * it into the residual, clears the component list, retained list, iteration
 * counter and totals and finds the first peak.  If psf is not NULL it is
 * copied too and the beam (alpha_b, omega_b) is fitted again (Sect. 3);
 * otherwise the beam is kept.  The noise level is kept.  *_on_host: 1 for
 * host memory, 0 for device memory. */
asp_status asp_reset(asp_ctx* ctx, const float* dirty, int dirty_on_host, const float* psf, int psf_on_host);

/* Per-kernel timing.  While on, minor cycles launch kernels directly (no CUDA
 * graph) and every launch is bracketed by CUDA events on the context stream;
 * asp_get_kernel_times reports per-kernel launches and total milliseconds
 * since profiling was switched on.  Switching resets the totals. */
typedef struct { char name[32]; int64_t launches; double total_ms; } asp_kernel_time;
asp_status asp_set_profiling(asp_ctx* ctx, int on);
asp_status asp_get_kernel_times(asp_ctx* ctx, asp_kernel_time* out, int cap, int* n);
/* Kernels this context has launched (graph replays counted per kernel node). */
asp_status asp_launch_count(asp_ctx* ctx, int64_t* n);

/* Allocation-free joint LM fit.  The paper has no counterpart: this is a
 * service for callers that cannot create device allocations of their own --
 * code running inside another framework's memory pool (the pool owns the
 * device memory budget), real-time pipelines that forbid allocation after
 * start-up (cudaMalloc can synchronise the device and take milliseconds), and
 * host threads that may run while another thread captures a CUDA graph in
 * global mode, where cudaMalloc is an illegal call.
 *
 * It fits n Gaussians (asp_gauss rows, host memory) to the FP32 image
 * image_dev (H x W, device, row-major) exactly as asp_fit_active_set does
 * (window = bounding box of the members' boxes, clipped; the last n_old
 * members' initial Gaussians are added back to the target; trial widths must
 * exceed omega_min, e.g. 0.25 omega_b; LM settings lm_lambda0, lm_rtol,
 * lm_xtol and lm_max_iter taken from *lm), writes the fitted rows to out
 * (host) and the outcome to info (host, may be NULL), and synchronises
 * stream.  No context, no cudaMalloc, cudaFree or allocating library call:
 * its device scratch is one file-scope __device__ array of
 * ASP_STATIC_SCRATCH_BYTES that every GPU loading the library holds until the
 * process exits.  Limits: n <= ASP_STATIC_KMAX (else ASP_ERR_UNSUPPORTED), at
 * most ASP_STATIC_GRID_MAX CTAs, and a window small enough for their shared
 * memory (ASP_STATIC_GRID_MAX x 12288 pixels; else ASP_ERR_UNSUPPORTED).
 * The first call on a device looks up the array's device address and sets
 * the kernel's shared-memory attribute (once per device; make that first call
 * before any stream capture).  All calls on a device share the array and it
 * keeps the last call's contents: each call clears what must start at zero,
 * and calls that overlap on the GPU (other threads or streams) race. */
#define ASP_STATIC_KMAX 8
#define ASP_STATIC_GRID_MAX 32
#define ASP_STATIC_SCRATCH_BYTES 5964032
asp_status asp_fit_static(const float* image_dev, int H, int W, const asp_gauss* init, int n, int n_old,
                          double omega_min, const asp_params* lm, asp_gauss* out, asp_fit_info* info,
                          void* stream);

/* Measured issue rates of the two pipes the LM pixel pass (Eq. 6 model,
 * Jacobian and normal equations) runs on, for its ALU roofline: FP32 fused
 * multiply-add (scalar, and Blackwell's packed two-lane fma.rn.f32x2) and
 * the MUFU ex2 unit, each from one full wave of independent dependency
 * chains on every SM of the current device, timed by CUDA events on the
 * legacy default stream (synchronised), with the SM clock each ran at
 * (clock64 cycles over event time).  Allocates and frees a few bytes of
 * scratch.  The paper has no counterpart: it is the measuring rod of the
 * roofline fractions the benchmark reports. */
typedef struct {
    int32_t sms;
    int32_t reserved;
    double fp32_fma_tflops;    /* scalar FP32 FMA, 2 flops each, whole device */
    double fp32_fma2_tflops;   /* packed two-lane FP32 FMA, 2 flops per lane */
    double ex2_gops;           /* ex2.approx.ftz.f32 results per second (1e9) */
    double sm_mhz_fma, sm_mhz_fma2, sm_mhz_ex2;     /* SM clock during each kernel */
    double fma_per_sm_clk, fma2_per_sm_clk, ex2_per_sm_clk;   /* per SM and clock */
} asp_alu_peaks;
asp_status asp_measure_alu_peaks(asp_alu_peaks* out);

/* Checkpoint the whole minor-cycle state (residual included) to a file, or
 * restore it into a context of the same size. */
asp_status asp_save_state(asp_ctx* ctx, const char* path);
asp_status asp_load_state(asp_ctx* ctx, const char* path);

/* ---------------------------------------------------------------- batches
 * Many independent images -- each with its own size, PSF, dirty image and
 * minor-cycle state -- advanced together.  The paper runs one image at a
 * time and has no batch of its own; its test data are 32-channel wide-band
 * observations (Sect. 4), and channels or fields imaged separately are
 * independent minor cycles, which this serves.  One minor-cycle iteration of
 * the whole batch is one
 * launch per kernel of the iteration with the images on grid.y, and the LM
 * fits (Eq. 6) of all images run in ONE cooperative launch in which image i
 * owns a group of CTAs (sized on the device each iteration from its fit
 * window and the policy the autotuner chose) with its own grid barrier.
 * asp_batch_minor_cycle
 * captures eight batch iterations into a CUDA graph and replays it.
 *
 * Every image's result is exactly what a context of its own would compute
 * (same kernels, same per-image buffers), given the same fit-group size. */
typedef struct asp_batch asp_batch;

typedef struct {
    int px_per_cta;        /* chosen LM window tile: target pixels per CTA (0: automatic rule) */
    int share_policy;      /* 0: equal CTA groups, 1: proportional to image area, 2: on demand each iteration */
    int n_candidates;      /* candidates timed */
    double best_ms;        /* time of the chosen candidate over the trial iterations */
    double default_ms;     /* time of the untuned setting (px_per_cta 0, equal groups) */
} asp_batch_tuning;

/* Create a batch of n images (1 <= n <= 152): image i is H[i] x W[i], its
 * dirty image dirty[i] (H x W) and PSF psf[i] (2H x 2W, zero lag at
 * [H, W]), FP32 row-major, all in host memory if on_host else device memory
 * (copied; the caller keeps ownership).  Every image gets its own context
 * (asp_init: beam fit, noise level) with the shared params and the batch's
 * stream (NULL: the legacy default stream).  Errors: ASP_ERR_INVALID_ARG
 * (bad n, size or pointer), ASP_ERR_UNSUPPORTED (more images than fit CTAs),
 * ASP_ERR_OOM, ASP_ERR_CUDA, or an image's asp_init error.  On error nothing
 * is left allocated. */
asp_status asp_batch_create(const asp_params* params, int n, const int* H, const int* W,
                            const float* const* dirty, const float* const* psf, int on_host, void* stream,
                            asp_batch** out);
asp_status asp_batch_destroy(asp_batch* b);
/* Restart every image from its dirty image (state, components and history
 * cleared; beam and noise level kept). */
asp_status asp_batch_reset(asp_batch* b);
/* Run up to n_iter more minor-cycle iterations on every image (an image
 * stops early on its own noise test).  stats: NULL or n entries (host),
 * filled per image as asp_minor_cycle fills its one.  Synchronises. */
asp_status asp_batch_minor_cycle(asp_batch* b, int n_iter, asp_cycle_stats* stats);
/* Autotuner of the batched fit: times n_trial_iter batch iterations from a
 * reset for each candidate window tile (pixels per CTA) and CTA-group
 * policy, keeps the fastest, and resets the batch.  out (host) may be NULL. */
asp_status asp_batch_autotune(asp_batch* b, int n_trial_iter, asp_batch_tuning* out);
/* Learned initial values for every image of the batch (as asp_set_mlp
 * for a context; one tensor-core inference per iteration covers all
 * images). */
asp_status asp_batch_set_mlp(asp_batch* b, const float* params_host, int enable);
/* Borrow image i's context for queries (residual, components, history,
 * stats, state); owned by the batch -- do not destroy it. */
asp_status asp_batch_image(asp_batch* b, int i, asp_ctx** ctx);
/* Kernels the batch has launched (graph nodes counted per replay). */
asp_status asp_batch_launch_count(asp_batch* b, int64_t* n);

/* Work queue over the batch's images: every image runs n_iter iterations
 * of its own minor cycle (its context's CUDA graph; the same kernels and
 * the same per-image results as asp_minor_cycle), so images advance
 * independently and a small image never waits for a large image's fits.
 * The images go longest first (by pixels) onto the least-loaded of n_lanes
 * CUDA streams, each lane running its images back to back; the call
 * synchronises once.  Each image's fit grid is capped at ceil(SMs /
 * n_lanes) CTAs so that the lanes' cooperative fits run side by side, and
 * px_per_cta > 0 sets the images' fit window tile (0: their parameters');
 * both change only the FP32 summation order of the fits, and stay set on
 * the images' contexts until the next call with other values (n_lanes = 1
 * and px_per_cta = 0 restore the uncapped defaults).  stats (host, n
 * entries, may be NULL) as asp_batch_minor_cycle.  Not with learned
 * initial values (ASP_ERR_UNSUPPORTED). */
asp_status asp_batch_run_queue(asp_batch* b, int n_iter, int n_lanes, int px_per_cta, asp_cycle_stats* stats);

/* Joint wide-band fit: the batch's images as the C channels of one
 * observation (the paper's data is multi-channel, Sect. 4; its fits are per
 * image).  A joint member has a centre (x, y) and an intrinsic width s
 * shared by every channel and an image-plane amplitude a_c per channel; in
 * channel c it is Eq. 6's Gaussian a_c exp(-r^2 / (2 w_c^2)) with w_c^2 =
 * s^2 + omega_b_c^2 (Eq. 7 with channel c's beam).  chi^2 is the sum over
 * channels of Eq. 6 over one shared window (the union of the members' boxes
 * of their widest convolved width), the target of channel c its residual
 * with the last n_old members of init added back.  LM rules of
 * asp_fit_active_set; trial centres inside the window and every w_c at most
 * the window extent.  init and out (host): n rows of 3 + C doubles (x, y,
 * s, a_1 .. a_C).  flux (host, may be NULL): n x C doubles, Eq. 8 per
 * channel, F_c = a_c w_c^2 / (alpha_b_c omega_b_c^2); is_point (host, may
 * be NULL): n ints, s^2 <= 1e-3 min_c omega_b_c^2.  Every image must have
 * the same size; n (3 + C) <= 4 x ASP_KMAX (ASP_ERR_UNSUPPORTED beyond).
 * The first call allocates its buffers (C x H x W floats of targets). */
asp_status asp_batch_fit_joint(asp_batch* b, const double* init, int n, int n_old, double* out, double* flux,
                               int* is_point, asp_fit_info* info);

/* ---------------------------------------------------------------- learned initial values
 * A 1024-256-256-4 GELU network proposes a new component's starting point
 * (amplitude / R(p*), log(omega / omega_b), x - x*, y - y*) from the 32 x 32
 * residual patch at the plain method's peak p*.  The paper has no learned
 * part: its initial values are the peak (simple method) or the peak of
 * smoothed residuals (Sect. 2 step 1, Sect. 3); the network only changes
 * where LM starts -- the active set and fit window still come from the
 * plain method, and a worse learned fit falls back to the plain start.
 *
 * The tensor-core product used for the network's wide layers, exposed for
 * tests: C[M x N] (FP32, row-major, ldc) = A[M x K] x B[N x K]^T with A and
 * B BF16 row-major (lda, ldb elements), all device pointers.  M % 128 == 0,
 * N % 256 == 0, K % 64 == 0, lda, ldb multiples of 8 and >= K, ldc a
 * multiple of 4 and >= N, 16-byte aligned bases; else ASP_ERR_INVALID_ARG.
 * Synchronises stream; ASP_ERR_TIMEOUT if a tensor-core wait ran out. */
asp_status asp_mlp_gemm(const void* A_dev, int lda, const void* B_dev, int ldb, float* C_dev, int ldc, int M, int N,
                        int K, void* stream);

/* Trainer of the network.  Parameters are one FP32 vector (host order
 * W1 [256 x 1024 row-major], b1 [256], W2 [256 x 256], b2 [256], W3 [4 x 256],
 * b3 [4]; asp_mlp_num_params gives its length).  The trainer keeps FP32
 * master weights and Adam moments on the device, BF16 copies of W1 and W2
 * for the tensor-core products, a data set and the scratch of a batch of up
 * to max_batch rows (rounded up to 128).  All host arrays are copied; the
 * trainer owns its device memory.  Errors: ASP_ERR_INVALID_ARG, ASP_ERR_OOM,
 * ASP_ERR_CUDA, ASP_ERR_TIMEOUT (a tensor-core wait ran out). */
typedef struct asp_mlp asp_mlp;
asp_status asp_mlp_num_params(long long* n);
asp_status asp_mlp_create(const float* params_host, int max_batch, void* stream, asp_mlp** out);
asp_status asp_mlp_destroy(asp_mlp* m);
/* Training set: n patches (n x 1024, host FP32, stored as BF16) and targets
 * (n x 4, host FP32). */
asp_status asp_mlp_set_data(asp_mlp* m, const float* X_host, const float* T_host, long long n);
/* Forward and backward pass (mean squared error) on data rows idx_host[0 ..
 * bn) (bn <= max_batch); with update != 0 one Adam step (learning rate lr,
 * beta1 0.9, beta2 0.999, eps 1e-8).  loss_out (1 float) and grads_out
 * (num_params floats, parameter order) are host pointers and may be NULL.
 * Synchronises. */
asp_status asp_mlp_step(asp_mlp* m, const int* idx_host, int bn, float lr, int update, float* loss_out,
                        float* grads_out);
/* Outputs (n x 4, host) for patches X_host (n x 1024, host), n <= max_batch. */
asp_status asp_mlp_predict(asp_mlp* m, const float* X_host, int n, float* Y_host);
asp_status asp_mlp_get_params(asp_mlp* m, float* params_host);

/* Learned initial values in a context's minor cycle.  params_host: the
 * network's FP32 parameter vector (order as above), copied; enable = 0
 * switches the proposals off again.  With it on, each iteration:
 *   1. the plain method (peak or smoothed peak, Sect. 2 step 1, Sect. 3)
 *      picks p*, the active set and the fit window as without it;
 *   2. the network maps the 32 x 32 patch of R at p* (divided by |R(p*)|)
 *      to (a0 / R(p*), log(omega0 / omega_b), x0 - x*, y0 - y*) -- BF16
 *      tensor-core products -- and LM starts the new member there (kept
 *      plain if the proposal is outside the window, not finite or below the
 *      width bound);
 *   3. fallback: if that fit ends non-finite or at the width bound, or ends
 *      with a chi^2 above chi^2 at the plain start point, LM is run again
 *      from the plain start and the better chi^2 is kept.
 * Both fits use the same window and members, so their chi^2 compare. */
asp_status asp_set_mlp(asp_ctx* ctx, const float* params_host, int enable);
/* Training-data harvest: while set, iteration t of the minor cycle writes
 * the 32 x 32 patch at the plain peak (1024 floats, divided by |R(p*)|) to
 * patches_dev + 1024 t and (a / R(p*), log(omega / omega_b), x - x*,
 * y - y*, R(p*), x*, y*, LM status) of the converged new member to
 * targets_dev + 8 t, for t < capacity (device pointers owned by the caller;
 * NULL patches_dev switches the harvest off). */
asp_status asp_set_harvest(asp_ctx* ctx, float* patches_dev, float* targets_dev, int capacity);

#ifdef __cplusplus
}
#endif

#endif /* ASP_H */
