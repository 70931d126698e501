/*
 * mbir.h -- C ABI of the GB300 model-based iterative reconstruction library for
 * spectral-domain OCT (Mason et al., "Model-based iterative reconstruction for
 * spectral-domain optical coherence tomography").
 *
 * The library applies the ISAM system operator Phi (Sec. 2.1, Eq. for_model),
 * its adjoint Phi^H (Sec. 2.1, Eq. back_model, taken as the exact transpose in
 * the real inner products) and solves
 *
 *     x = argmin_x 1/2 ||Phi(x) - y||_2^2 + lambda ||Psi x||_1     (Eqs. obj, ls_obj)
 *
 * with FISTA (Sec. 2.3, Eq. alg), Psi = I or an orthonormal Daubechies wavelet
 * (Sec. 2.2).  Every step runs in CUDA kernels on one GPU.
 *
 * Conventions shared by all calls
 * -------------------------------
 *  Image x      complex, row-major [nx][nz]: nx A-scans (lateral pixel dx_um),
 *               nz depth pixels (dz_um, zero delay at n = 0), depth contiguous.
 *               Interleaved (re, im) float32 pairs for MBIR_FP32*,
 *               float64 pairs for MBIR_FP64.
 *  Measurements y  real, row-major [nx][m]: m spectrometer pixels at the
 *               wavenumbers k[m] of the geometry.  float32 (MBIR_FP32*) or
 *               float64 (MBIR_FP64).
 *  Mask         uint8 [nx][m], 1 = measured, 0 = not measured (diag(s) of
 *               Eq. for_model); NULL means every sample is measured.  Values of
 *               y where the mask is 0 are ignored.
 *  Pointers     x, y, mask are DEVICE pointers owned by the caller.  The plan owns
 *               its device tables and workspace.  Calls are asynchronous on the
 *               given cudaStream_t (passed as void*, NULL = legacy default stream)
 *               unless stated otherwise.
 *  Errors       every call returns an mbir_status; no call aborts, traps or
 *               exits.  Arguments are validated on the host before any launch.
 *               MBIR_ERR_CUDA reports a failed CUDA runtime call (the CUDA error
 *               text is kept, see mbir_last_error).
 *  Threads      a plan may be used from one host thread at a time; calls on
 *               different plans are independent.
 */
#ifndef MBIR_H
#define MBIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mbir_plan_s* mbir_plan;

typedef enum {
  MBIR_OK = 0,
  MBIR_ERR_INVALID = -1,          /* bad argument (NULL, non-positive size, non-finite value) */
  MBIR_ERR_UNSUPPORTED_SIZE = -2, /* size outside what the kernels handle (see mbir_plan_create) */
  MBIR_ERR_OOM = -3,              /* device allocation failed */
  MBIR_ERR_CUDA = -4,             /* a CUDA runtime call failed */
  MBIR_ERR_TIMEOUT = -5,          /* a bounded device-side wait gave up */
  MBIR_ERR_NOT_CONVERGED = -6     /* solver stopped at max_iter before rel_tol was met */
} mbir_status;

typedef enum { MBIR_FP32 = 0, MBIR_FP32_COMPENSATED = 1, MBIR_FP64 = 2 } mbir_precision;

/* MBIR_PENALTY_TV: the isotropic total variation of Sec. 2.2 (single-scan solves and
 * the prox entry points; the batch and serving paths take L1 and DB4 only). */
typedef enum { MBIR_PENALTY_L1 = 0, MBIR_PENALTY_DB4 = 1, MBIR_PENALTY_TV = 2 } mbir_penalty;

/* Back-projection used for the gradient (single-scan solves only):
 * MBIR_BACKPROJ_TRANSPOSE  the exact transpose Phi^H of mbir_adjoint;
 * MBIR_BACKPROJ_HILBERT    the paper's Phi* of mbir_adjoint_hilbert (Eq. back_model). */
typedef enum { MBIR_BACKPROJ_TRANSPOSE = 0, MBIR_BACKPROJ_HILBERT = 1 } mbir_backprojection;

/*
 * Optical geometry of one B-scan (Sec. 2.1).  Host memory; copied by
 * mbir_plan_create, so the caller may free it afterwards.
 *
 *  nx, nz, m    A-scans, depth pixels, spectrometer pixels.
 *  k            host [m] wavenumbers (rad/um), strictly monotone.
 *  source       host [m] source amplitude A(k) >= 0, or NULL for A = 1.
 *  dx_um        lateral pixel; lateral frequencies q_l = 2 pi l~/(nx dx), l~ the
 *               signed FFT index (Eq. 4).
 *  dz_um        depth pixel; 0 selects pi / (2 nz max|dk|), the positive twin-free
 *               half of the resolved depth range (the role of Q, Eq. for_model).
 *  na, z_focus_um  Gaussian beam filter G(q,k) = exp(-q^2 / (2 k^2 na^2)) focused
 *               at depth z_focus (the ISAM filter f^ of Eq. 5); na <= 0 gives G = 1.
 *  disp_a, disp_b, k0  dispersion phase Omega = a (k-k0)^2 + b (k-k0)^3 (Sec. 2.1).
 *  falloff_half_um  depth falloff w(z) = exp(-ln2 (z/z_half)^2); <= 0 disables.
 *  kb_width     Kaiser-Bessel interpolation width J (even, 4..8) of the NUFFT that
 *               realises the ISAM resampling (Sec. 2.1, "u = Kx").
 *  kb_oversamp  axial oversampling sigma; K = sigma * nz must be an integer.
 *               Only 2.0 is supported.
 *  kb_alpha     KB shape; 0 selects 2.34 * J.
 *  precision    mbir_precision of x and y for every call on the plan.
 */
typedef struct {
  int32_t nx, nz, m;
  const double* k;
  const double* source;
  double dx_um, dz_um;
  double na, z_focus_um;
  double disp_a, disp_b, k0;
  double falloff_half_um;
  int32_t kb_width;
  double kb_oversamp;
  double kb_alpha;
  int32_t precision;
} mbir_geometry;

/*
 * Solver options (Sec. 2.3).
 *  penalty            mbir_penalty: l1 on pixels (Psi = I), on the 3-level periodic
 *                     orthonormal Daubechies wavelet with 4 vanishing moments, or the
 *                     isotropic total variation (TV) of Sec. 2.2.
 *  lambda             penalty weight; if lambda_is_relative != 0 the weight used is
 *                     lambda * max|Psi Phi^H(s y)| (one extra adjoint at set-up; for TV
 *                     the pixel maximum max|Phi^H(s y)|, as for l1).
 *  max_iter           FISTA iterations (>= 1).
 *  min_iter, rel_tol  if rel_tol > 0 the solve stops after iteration k >= min_iter
 *                     once |F(z^{k-1}) - F(z^{k-2})| <= rel_tol * F(z^{k-2}); the
 *                     objective is then read back every iteration (a host sync).
 *  power_iters        power iterations for L = lambda_max(Phi^H Phi) when step <= 0.
 *  step               gradient step delta; <= 0 selects 1 / (1.01 L).
 *  warm_start         != 0: start from the x passed in instead of 0.
 *  tv_iters           TV only: dual projected-gradient (FGP) steps per prox, from the
 *                     zero dual at every prox; <= 0 selects 20.
 *  backprojection     mbir_backprojection of the gradient step.  With
 *                     MBIR_BACKPROJ_HILBERT the step bound L is the power iteration's
 *                     estimate for Phi* Phi and the relative lambda uses Phi*(s y);
 *                     the spectrometer length m must then be a product of 2, 3, 5, 7
 *                     and at most 8192 (else MBIR_ERR_UNSUPPORTED_SIZE).
 */
typedef struct {
  int32_t penalty;
  double lambda;
  int32_t lambda_is_relative;
  int32_t max_iter;
  int32_t min_iter;
  double rel_tol;
  int32_t power_iters;
  double step;
  int32_t warm_start;
  int32_t tv_iters;
  int32_t backprojection;
} mbir_solve_opts;

/*
 * Solver report (host memory, filled by mbir_solve).
 *  iters             iterations run.
 *  status            mbir_status of the solve.
 *  objective         F(z) of the returned iterate (FP64 on the device).
 *  lipschitz         L used (0 when step was given).
 *  step, lambda_used the delta and the absolute lambda used.
 *  objective_trace   optional host array of trace_len doubles; entry k-1 receives
 *                    F(z^{k-1}) measured during iteration k (NULL: not recorded; the
 *                    per-iteration objective is then only reduced when rel_tol > 0).
 */
typedef struct {
  int32_t iters;
  int32_t status;
  double objective;
  double lipschitz;
  double step;
  double lambda_used;
  double* objective_trace;
  int32_t trace_len;
} mbir_solve_info;

/*
 * Build a plan for one geometry: validates it, derives the FP64 tables (lateral
 * frequencies, beta = sqrt(4k^2 - q^2) grid positions, filter, deapodisation,
 * KB kernel, FFT twiddles) on the host and uploads them, and allocates the
 * workspace, on the current CUDA device.  Synchronous.
 * Supported sizes: nz in [8, 4096] with every prime factor <= 7 (K = 2 nz); nx
 * in [2, 4096]; nx * nz and nx * m below 2^31; m in [1, 65536].  A width nx with
 * a prime factor above 7 runs its lateral transform (Eq. 4) in the Bluestein
 * (chirp-z) form, a convolution through transforms of the smallest length
 * L >= 2 nx - 1 whose prime factors are <= 7; L must be at most 4096, which
 * admits every width up to 2048 (wider ones return MBIR_ERR_UNSUPPORTED_SIZE).
 * Returns MBIR_ERR_INVALID / MBIR_ERR_UNSUPPORTED_SIZE before touching the GPU.
 * stream: used for the uploads; *out receives the plan (NULL on failure).
 */
int mbir_plan_create(const mbir_geometry* geometry, void* stream, mbir_plan* out);

/* Free a plan and its device memory (synchronises the device).  NULL is a no-op. */
void mbir_plan_destroy(mbir_plan plan);

/* Geometry sizes of a plan; any output pointer may be NULL. */
int mbir_plan_dims(mbir_plan plan, int32_t* nx, int32_t* nz, int32_t* m, int32_t* precision);

/*
 * A plan for a 3-D volume: the B-scan geometry plus a second lateral axis of ny
 * pixels spaced dy_um (<= 0 selects dx_um), the volumetric acquisition of
 * Sec. 3.1 with the operator of Sec. 2.1 over both lateral axes: the lateral
 * Fourier transform of Eq. 4 is 2-D, and the ISAM resampling of Eq. 5 and the
 * beam filter see |q|^2 = q_x^2 + q_y^2 with q_y = 2 pi l~_y / (ny dy).
 * Layouts: image x [nx][ny][nz] complex, measurements y and mask [nx][ny][m],
 * depth / spectrum contiguous.  A volume plan runs mbir_forward and mbir_adjoint
 * (same arguments, these layouts) and mbir_solve with the l1 penalty (see there);
 * the other calls that take a plan return MBIR_ERR_UNSUPPORTED_SIZE for it.  Sizes: ny in [2, 4096] with the same rule as
 * nx (Bluestein beyond 7-smooth), nx * ny * nz and nx * ny * m below 2^31; the
 * other limits as mbir_plan_create.  The resampling table has one row per
 * (|lx|, |ly|): (nx/2 + 1)(ny/2 + 1) m entries of 16 bytes (FP32), built on the
 * host.  Returns MBIR_ERR_INVALID for ny < 2.  Synchronous.
 */
int mbir_volume_plan_create(const mbir_geometry* geometry, int32_t ny, double dy_um, void* stream,
                            mbir_plan* out);

/* The second lateral size of a plan (1 for a B-scan plan). */
int mbir_volume_dims(mbir_plan plan, int32_t* ny);

/*
 * y = Phi(x) (Eq. for_model): lateral FFT, KB-NUFFT resampling onto
 * beta = sqrt(4k^2 - q^2) (Eq. 5), filter, dispersion phase, inverse lateral FFT,
 * real part, mask.  x: device [nx][nz] complex; y: device [nx][m] real, fully
 * written (0 where the mask is 0).  Uses the plan's workspace: calls on one plan
 * must be ordered (same stream, or synchronised).
 */
int mbir_forward(mbir_plan plan, const void* x, const uint8_t* mask, void* y, void* stream);

/*
 * x = Phi^H(y) (Eq. back_model as the exact transpose of mbir_forward in the
 * real inner products <a,b> = Re sum conj(a) b).  y: device [nx][m] real (entries
 * with mask 0 ignored); x: device [nx][nz] complex, fully written.
 */
int mbir_adjoint(mbir_plan plan, const void* y, const uint8_t* mask, void* x, void* stream);

/*
 * x = Phi*(y) = K^H Q^T D^H diag(e^{-j Omega}) A(s y), the paper's back-projection
 * (Sec. 2.1, Eq. back_model), with A(r) = r - j d H(r) the conjugate analytic
 * signal along the spectrometer axis of each A-scan: H is the discrete Hilbert
 * transform (DFT multiplier -j sgn(f), zero at DC and at the Nyquist bin), d = +1
 * when the plan's wavenumbers increase with the pixel index (as printed) and
 * d = -1 when they decrease (the side on which the model's e^{-j 2 k z} lies).
 * The mask is applied before A.  On measurements whose A-scans are one-sided
 * along m, Phi* = 2 Phi^H; in general the two differ (dispersion, edges).
 * y: device [nx][m] real; x: device [nx][nz] complex, fully written.  Uses the
 * plan's workspace; builds the m-point transform tables on the first call
 * (synchronous then).  m must be a product of 2, 3, 5, 7 and at most 8192, else
 * MBIR_ERR_UNSUPPORTED_SIZE.
 */
int mbir_adjoint_hilbert(mbir_plan plan, const void* y, const uint8_t* mask, void* x, void* stream);

/*
 * The paper's baseline (Sec. 3, "direct ISAM on linearly interpolated
 * measurements"): every unmeasured sample of an A-scan is filled by linear
 * interpolation in the spectrometer pixel index between the nearest measured
 * samples on either side (the nearest measured value is held before the first and
 * after the last one; an A-scan without a measured sample stays zero), then
 * x = Phi*(y_interp) as in mbir_adjoint_hilbert with every sample counted as
 * measured.  mask NULL: no interpolation.  Same layouts, sizes and errors as
 * mbir_adjoint_hilbert (the interpolation needs twice its shared memory: FP64
 * plans take m <= 4096).
 */
int mbir_isam_interpolated(mbir_plan plan, const void* y, const uint8_t* mask, void* x, void* stream);

/*
 * Normalised cross-correlation of magnitudes (Sec. 3, Eq. ncc):
 *   r = sum (|x_i| - mean|x|)(|z_i| - mean|z|) / sqrt(sum (|x_i| - mean|x|)^2 sum (|z_i| - mean|z|)^2)
 * over the plan's [nx][nz] images x and z (device, complex, plan precision).
 * Two passes (means, then centred sums), FP64 accumulation in a fixed order.
 * *r (host) is 0 when either image has constant magnitude.  Synchronous.
 */
int mbir_ncc(mbir_plan plan, const void* x, const void* z, double* r, void* stream);

/*
 * Golden-section search of the penalty weight (Sec. 3: lambda chosen to maximise
 * the NCC with the ground truth).  t = log10 of the relative lambda (the weight is
 * 10^t * max|Psi Phi^H(s y)|, or Phi* with MBIR_BACKPROJ_HILBERT) is searched in
 * [log10_lo, log10_hi] with n_eval >= 2 evaluations: interior points
 * c = b - g (b - a), d = a + g (b - a), g = (sqrt 5 - 1)/2; while evaluations
 * remain, f(c) >= f(d) keeps [a, d], else [c, b]; one new point per step.  Each
 * evaluation is an mbir_solve with opts (lambda and lambda_is_relative are
 * replaced; the first evaluation derives the step when opts->step <= 0 and every
 * later one reuses it) followed by mbir_ncc against z_true.  x (device [nx][nz])
 * receives the reconstruction of the best evaluation (the first one on ties).
 * Synchronous.  Allocates one image of scratch for the duration of the call.
 */
typedef struct {
  double lambda_rel;         /* best 10^t */
  double lambda;             /* absolute weight used there */
  double ncc;                /* its NCC */
  double step;               /* gradient step used by every evaluation */
  int32_t evaluations;
  double* trace_lambda_rel;  /* optional host [n_eval]: evaluated 10^t in order (NULL: not recorded) */
  double* trace_ncc;         /* optional host [n_eval]: their NCC */
} mbir_lambda_search_info;

int mbir_lambda_search(mbir_plan plan, const void* y, const uint8_t* mask, const void* z_true,
                       const mbir_solve_opts* opts, double log10_lo, double log10_hi, int32_t n_eval, void* x,
                       mbir_lambda_search_info* info, void* stream);

/*
 * FISTA (Eq. alg) from x^1 = z^0 = 0 (or the x passed in when warm_start),
 * t^1 = 1, for opts->max_iter iterations (or until rel_tol), writing z^k to x.
 * Allocates the iteration state on the first call for a given plan and keeps it.
 * Synchronous when it has to read a device scalar back (step or lambda derived on
 * the device, rel_tol > 0, or info != NULL); otherwise asynchronous on stream.
 * On a volume plan (mbir_volume_plan_create) the image and measurements take the
 * volume layouts and the options are restricted to the l1 penalty, the transpose
 * back-projection and a fixed iteration count (rel_tol = 0; MBIR_ERR_INVALID
 * otherwise; the objective trace is not recorded).  Each iteration is one volume
 * Phi, one volume Phi^H and two elementwise passes (no fused solver passes).
 */
int mbir_solve(mbir_plan plan, const void* y, const uint8_t* mask, const mbir_solve_opts* opts,
               void* x, mbir_solve_info* info, void* stream);

/*
 * FISTA on n B-scans at once (the uneven-size batch): plans[i] (each plan at most
 * once, all with the same precision, KB width and shape), y[i], mask[i] (mask may
 * be NULL, or mask[i] NULL), opts[i] and x[i] as for mbir_solve.  Scans whose row
 * kernels alone give every SM at least three CTAs (nx/2 + 1 >= 3 x the SM count)
 * run the single-scan path of mbir_solve; for the others every stage of the path
 * -- power iteration, lambda rule, the operator passes, the FISTA epilogues and
 * the wavelet levels -- is one launch over all of them, and their iteration loop
 * is captured into a CUDA graph and replayed.  When `stream` is a created stream
 * (not the legacy or per-thread default) and both kinds are present, the wide
 * scans run on a high-priority stream and the shared stages on a second stream,
 * both forked from `stream` and joined back to it, so that the shared stages fill
 * the SMs the wide scans' launches leave idle.  Each scan's result does not
 * depend on what it is batched with (a wide scan's equals its mbir_solve result).  All opts[i].max_iter must be equal,
 * rel_tol must be 0 (fixed iteration count), the penalty l1 or db4 and the
 * back-projection the transpose.  info (NULL or n entries) receives
 * iters, lipschitz, step and lambda_used; objective is not evaluated (NaN).
 * Synchronous at set-up (one read-back for the shared scans, and the read-backs
 * of mbir_solve for each wide scan) and when info != NULL.
 */
int mbir_solve_batch(mbir_plan* plans, int32_t n, const void* const* y, const uint8_t* const* mask,
                     const mbir_solve_opts* opts, void* const* x, mbir_solve_info* info, void* stream);

/*
 * Serving with continuous batching.  Requests (one B-scan solve each, on any plan
 * of one precision) are submitted at any time; each mbir_server_step is one tick:
 * pending requests are admitted in arrival order while the device state they
 * need (mbir_server_request_bytes) fits the HBM budget (a request larger than the
 * whole budget fails with MBIR_ERR_OOM), the newly admitted ones run their set-up
 * (power iteration, lambda rule) as one batch, every active request advances one
 * FISTA iteration in one batched pass, and requests that reached max_iter or
 * their relative-objective tolerance (rel_tol, after min_iter) are retired: z is
 * copied to their x and their state freed.  Iterates, momentum, step size and the
 * objective history stay on the device.  A request's result does not depend on
 * the other requests it shared ticks with.  y, mask and x of a request must stay
 * valid until it is done.  Requests take the l1 or db4 penalty and the transpose
 * back-projection.  Synchronous (each step waits for its work).
 */
typedef struct mbir_server_s* mbir_server;

int mbir_server_create(size_t hbm_budget_bytes, void* stream, mbir_server* out);
void mbir_server_destroy(mbir_server srv);
/* *ticket identifies the request in mbir_server_poll. */
int mbir_server_submit(mbir_server srv, mbir_plan plan, const void* y, const uint8_t* mask,
                       const mbir_solve_opts* opts, void* x, int64_t* ticket);
/* One tick; any output pointer may be NULL. */
int mbir_server_step(mbir_server srv, int32_t* n_active, int32_t* n_pending, int32_t* n_completed);
/*
 * *done = 1 once the request finished (its info then filled: iters, status --
 * MBIR_ERR_NOT_CONVERGED when rel_tol was not met by max_iter, MBIR_ERR_OOM when it
 * could never fit -- objective F(z^{k-1}) when rel_tol > 0, lipschitz, step,
 * lambda_used); *latency_s = seconds from submission to completion (or so far).
 * A finished ticket is released by the poll that reports it.
 */
int mbir_server_poll(mbir_server srv, int64_t ticket, int32_t* done, mbir_solve_info* info, double* latency_s);
int mbir_server_stats(mbir_server srv, size_t* bytes_in_use, size_t* peak_bytes, int64_t* completed);
/* Device bytes a request on `plan` holds while active. */
int mbir_server_request_bytes(mbir_plan plan, int32_t penalty, int32_t max_iter, size_t* bytes);

/*
 * Host-only replay of the server's admission rule (no GPU): request i arrives at
 * tick arrive_tick[i] (non-decreasing), needs bytes[i] and stays service_ticks[i]
 * ticks once admitted.  Fills admit_tick / done_tick (-1 for requests larger than
 * the budget) and the peak bytes held.
 */
int mbir_admission_simulate(size_t budget, int32_t n, const int64_t* bytes, const int32_t* arrive_tick,
                            const int32_t* service_ticks, int32_t* admit_tick, int32_t* done_tick,
                            int64_t* peak_bytes);

/*
 * lambda_max(Phi^H Phi) for this plan and mask by power iteration from a fixed
 * pseudo-random start (counter-based hash of the pixel index), FP64 norms
 * (step-size bound of Sec. 2.3).  Writes the estimate to *out (host).  Synchronous.
 */
int mbir_lipschitz(mbir_plan plan, const uint8_t* mask, int32_t iters, double* out, void* stream);

/*
 * Proximal map of tau * ||Psi x||_1 (Sec. 2.3): z = Psi^T soft(Psi v, tau) with
 * the complex soft-threshold c max(0, 1 - tau/|c|).  v, z: device [nx][nz]
 * complex (may alias).  penalty: mbir_penalty.  MBIR_PENALTY_DB4 needs nx and nz
 * divisible by 8 with nx/8, nz/8 >= 1 and nx/4, nz/4 >= 8.
 */
int mbir_prox(mbir_plan plan, int32_t penalty, const void* v, double tau, void* z, void* stream);

/*
 * Proximal map of tau * TV (Sec. 2.2-2.3): z = argmin 1/2 ||x - v||^2 + tau TV(x), TV the
 * isotropic total variation sum_ij sqrt(|x(i+1,j) - x(i,j)|^2 + |x(i,j+1) - x(i,j)|^2)
 * with the differences that would leave the image taken as zero.  Computed by
 * `iters` steps of fast gradient projection on the dual problem (the dual field p
 * holds one complex number per direction and pixel, |p1|^2 + |p2|^2 <= 1), from p = 0:
 *   p_k = project(r_k + grad(v + tau div r_k) / (8 tau)),  r_{k+1} = p_k + m_k (p_k - p_{k-1}),
 * with FISTA's momentum m_k, and z = v + tau div p_iters.  tau = 0 or iters <= 0 copy v.
 * v, z: device [nx][nz] complex, distinct.  mbir_prox with MBIR_PENALTY_TV uses 20
 * steps.  The plan keeps three dual fields (16 bytes a pixel each in FP32, 32 in FP64),
 * allocated on first use.
 */
int mbir_prox_tv(mbir_plan plan, const void* v, double tau, int32_t iters, void* z, void* stream);

/*
 * Orthonormal 3-level periodic 2-D wavelet analysis c = Psi x (inverse = 0) or
 * synthesis x = Psi^T c (inverse = 1), Mallat layout in the [nx][nz] array (at each
 * level the low-low block splits into [[LL, LH], [HL, HH]], first index lateral).
 * in, out: device [nx][nz] complex, distinct.
 */
int mbir_wavelet(mbir_plan plan, int32_t inverse, const void* in, void* out, void* stream);

/*
 * mbir_wavelet without a plan and without allocating: for callers that cannot
 * call cudaMalloc -- a real-time loop that must not allocate once running, an
 * embedding that hands the library only pre-sized buffers, or a process whose
 * device memory is owned by another allocator.  The paper has no counterpart;
 * this is a deployment convenience.
 *  nx, nz     image size; both divisible by 8 and >= 32, nx * nz <= 2^21
 *             (2097152 pixels, e.g. 1024 x 2048).  Larger sizes return
 *             MBIR_ERR_UNSUPPORTED_SIZE (see mbir_last_error).
 *  inverse    0: analysis c = Psi x; 1: synthesis x = Psi^T c (layout as mbir_wavelet).
 *  in, out    device [nx][nz] complex64, distinct, owned by the caller.
 * Scratch: a file-scope device array of 5 MiB + 256 bytes (the filter taps and
 * the level-1/2 low-low blocks) that every GPU loading the library holds until
 * exit; nothing in it needs to start at zero, since a call writes every element it
 * reads.  The array is placed in device memory when the library's module loads
 * into a context, which with CUDA's default lazy module loading is the first
 * call of the library there (this one or any other); make that first call at
 * start-up, before another allocator takes the device's memory.  A placement that
 * fails returns MBIR_ERR_CUDA with the reason in mbir_last_error.
 * All calls in a context share the array, so calls that overlap on the GPU (other
 * streams, other threads) race: order them.  The first call in a context sets up:
 * it looks up the array's device address for that context, sets the kernels'
 * attributes and writes the taps into the array, then synchronises the device;
 * make that first call before any stream capture.  Addresses are kept per CUDA
 * context handle (a device's primary context, or a context the caller made
 * current), up to 64 contexts.  A context made after cudaDeviceReset that happens
 * to reuse the old context's handle would keep the old address: do not reset the
 * device between calls.  Allocates nothing, ever.
 */
int mbir_wavelet_static(int32_t nx, int32_t nz, int32_t inverse, const void* in, void* out, void* stream);

/*
 * Launch-shape autotuner for a plan's shape class (batched and single-scan solves
 * alike; the paper, which ran Matlab on a CPU, has no counterpart).  Candidates:
 * the lateral tile width (columns per CTA, powers of two up to 16 within the
 * kernels' shared-memory tile), the order of the lateral radices, and the row
 * adjoint kernel (paired gather with per-term weights, paired gather, single-row gather,
 * shared-memory atomics, as far
 * as the plan can run each).  The lateral ones are timed first with the automatic
 * adjoint kernel, then the adjoint kernels with the best lateral choice.  Each
 * candidate is warmed once, then timed over `reps` forward + adjoint pairs on
 * synthetic data with CUDA events on `stream`.  The plan's current choice is timed
 * first and a candidate replaces the kept one only when it is at least 2 % faster
 * (choices within timing noise do not churn).  The kept one stays on the plan and is
 * recorded for the shape class (nx, nz, m, KB width, precision), and plans of that
 * class created later in the process start from it.  The choices only reorder
 * floating-point operations.
 *
 * Tune a plan before its first solve or server submission: a new tile width
 * resizes the solver's per-CTA partial-sum buffers, and the plan's own solver state
 * is dropped for that (request contexts made earlier would not be).  Allocates and
 * frees two scratch buffers; synchronises the stream.  *best receives the kept
 * tuning and its time, *n_tried the number of timed candidates (either may be NULL).
 */
typedef struct {
  int32_t tile_c;          /* lateral tile width, columns per CTA */
  int32_t lateral_order;   /* 0: largest radix first, 1: smallest radix first */
  int32_t adjoint_kernel;  /* 5: paired gather with per-term weights (two CTAs an SM), 4: paired gather,
                              1: single-row gather, 2: atomics, -1: automatic */
  double pair_ms;          /* measured forward + adjoint time (autotune), else 0 */
} mbir_tuning;

int mbir_plan_autotune(mbir_plan plan, int32_t reps, mbir_tuning* best, int32_t* n_tried, void* stream);
/* The plan's current launch choices (pair_ms = 0). */
int mbir_plan_get_tuning(mbir_plan plan, mbir_tuning* out);
/* Apply a tuning (e.g. one found for another plan of the same shape).  MBIR_ERR_INVALID
 * when a choice does not fit the plan; the same caveat as for mbir_plan_autotune. */
int mbir_plan_set_tuning(mbir_plan plan, const mbir_tuning* t);

/*
 * Kernel timing (tracing).  mbir_profile_begin makes every later launch on the plan
 * record a CUDA event pair on its stream (up to `capacity` launches; further
 * launches run unrecorded).  mbir_profile_end waits for the recorded events, fills
 * up to max_entries entries, one per kernel class that ran (static names), stops
 * recording and frees the events.  *n_entries receives the entry count.
 */
typedef struct {
  const char* name;      /* kernel class, e.g. "row_forward" */
  int64_t launches;      /* recorded launches */
  double total_ms;       /* summed event time */
} mbir_profile_entry;

int mbir_profile_begin(mbir_plan plan, int32_t capacity);
/* Between begin and end: record only launches of one kernel class (a name as
 * returned by mbir_profile_end), or of every class again with NULL.  Recording a
 * single class leaves the other launches undisturbed by event records, so a run
 * can be timed while one kernel's launch durations are taken.
 * MBIR_ERR_INVALID: no recording is active or the name is unknown. */
int mbir_profile_only(mbir_plan plan, const char* kernel_class);
int mbir_profile_end(mbir_plan plan, mbir_profile_entry* out, int32_t max_entries, int32_t* n_entries);

/* Static description of a status code. */
const char* mbir_status_string(int status);

/* Text of the last CUDA failure seen by this thread ("" if none). */
const char* mbir_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MBIR_H */
