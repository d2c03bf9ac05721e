/*
 * astrophot_gb300.h -- C ABI of the GB300 chi^2 forward-modelling path.
 *
 * The library renders the summed light of parametric sources onto pixel grids
 * with per-pixel Gauss-Legendre quadrature, convolves galaxy light with the
 * image PSF, and reduces the masked, variance-weighted chi^2 with its gradient
 * and the Levenberg-Marquardt normal equations, then takes damped LM steps.
 * The method is AstroPhot (Stone et al. 2023, arXiv:2308.01957); each entry
 * point cites the section of the paper that defines what it computes.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Device pointers ("_dev") are CUDA global-memory addresses on the context's
 *    device; host pointers ("_host") are ordinary CPU memory.  The caller owns
 *    every buffer it passes; the library owns only the scratch it allocates in
 *    ap_set_problem() and frees in ap_set_problem()/ap_destroy().
 *  - All work is enqueued on the caller's stream (cudaStream_t passed as void*;
 *    NULL = legacy default stream).  No call synchronises the host except
 *    ap_set_problem() (it uploads its plans), the first ap_eval_adaptive() or
 *    ap_get_adaptive_layout() (they build the adaptive plan), ap_get_status(),
 *    ap_get_error(), ap_get_state(), ap_get_timing() and the *_host outputs of
 *    ap_lm_iterate() / ap_lm_continue() / ap_eval_adaptive().  Arrays of
 *    device pointers passed from the host (ap_render's model_dev) are read
 *    during the call: they need not outlive it.
 *  - Every call returns AP_OK (0) or an AP_ERR_* code; none aborts or traps.
 *    ap_get_error() returns a one-line description of the last failure.
 *  - Images are row-major, pitch = W elements.  Pixel (i, j) (row i, column j)
 *    covers [j, j+1) x [i, i+1) in pixel coordinates; a pixel-coordinate point
 *    (u, v) sits at world position origin + A (u, v) (the "pixel scale
 *    matrix" of the paper's multi-band example; coordinates "from the bottom
 *    corner" of its configuration example).  Row 0 is the bottom row.
 *  - theta is float64 in world units; PA in radians counter-clockwise from +x;
 *    intensities and fluxes linear.
 */
#ifndef ASTROPHOT_GB300_H
#define ASTROPHOT_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define AP_OK            0
#define AP_ERR_ARG       1   /* invalid argument or descriptor; nothing enqueued   */
#define AP_ERR_CUDA      2   /* a CUDA runtime call failed (message has the name)  */
#define AP_ERR_NOT_SPD   3   /* damped normal matrix not positive definite after
                                all lambda increases (per group, in the status)    */
#define AP_ERR_NONFINITE 4   /* variance <= 0 or non-finite on an unmasked pixel   */
#define AP_ERR_TIMEOUT   5   /* a bounded device loop gave up                      */
#define AP_ERR_STATE     6   /* call order: no problem set yet                     */
#define AP_ERR_NOMEM     7   /* device allocation failed                           */

/* ---- profile types (Sec. "A Zoo of Models"); slot order of theta per type */
#define AP_SERSIC      0   /* x0, y0, q, PA, n, Re, Ie                             */
#define AP_EXPONENTIAL 1   /* x0, y0, q, PA, Re, Ie      (Sersic with n = 1)       */
#define AP_GAUSSIAN    2   /* x0, y0, q, PA, sigma, F                              */
#define AP_MOFFAT      3   /* x0, y0, q, PA, n, Rd, F                              */
#define AP_SKY_FLAT    4   /* S          (per unit world area)                     */
#define AP_SKY_PLANE   5   /* S, gx, gy  (S + gx (x - xc) + gy (y - yc))           */
#define AP_PSF_STAR    6   /* x0, y0, F: a point source drawn with its image's PSF
                              image (normalised) as a pixel map, interpolated
                              bilinearly between the map's pixel centres on the
                              image's pixel grid, its centre pixel on (x0, y0);
                              never convolved; needs an image with a PSF       */

/* ---- arithmetic of the path ---------------------------------------------- */
#define AP_PREC_MIXED  0   /* render, convolution, Jacobian in float32; chi^2,
                              gradient partials, b_n, normal-matrix sums and the
                              LM solve in float64                                 */
#define AP_PREC_F64    1   /* every step in float64 (the plain FP64 GPU form)    */

typedef struct ap_ctx ap_ctx;

typedef struct {
  int precision;     /* AP_PREC_MIXED or AP_PREC_F64                            */
  int quad_order;    /* Q in 1..7: Gauss-Legendre order per pixel axis (Q^2
                        evaluations per pixel, Sec. "Pixel Integration")         */
  int device;        /* CUDA device ordinal                                     */
  int tile_w;        /* convolution tile width in pixels (0 = autotuned)        */
  int tile_h;        /* convolution tile height in pixels (0 = autotuned)       */
  int jcol_mode;     /* PSF convolution of the Jacobian columns (mixed form):
                        AP_JCOL_AUTO, AP_JCOL_DIRECT or AP_JCOL_FFT            */
  int conv_variant;  /* 0: correlation tile variant chosen by tile_w/tile_h or
                        autotuned; v >= 1 forces variant v - 1 of
                        ap_get_conv_variant() (AP_ERR_ARG from ap_set_problem
                        if it does not fit the problem's largest PSF)         */
  int gram_tc_min;   /* mixed form, J^T W J tile Grams: 0 = chosen by timing in
                        ap_set_problem; k >= 1: tiles with k .. 128 Jacobian
                        columns run on the tensor-core (tcgen05) kernel, the
                        others on the warp-MMA kernel (k > 128: none); k is
                        rounded up to 1 + a multiple of 16                     */
} ap_options;

/* Jacobian-column convolution modes.  AUTO times both on the problem in
   ap_set_problem and keeps the faster.  FFT (overlap-save blocks of 64^2 or
   128^2, PSFs up to 97 x 97) is the FFT convolution mode the paper names for
   large PSFs; it falls back to DIRECT when some convolved image's PSF is
   larger, and in the float64 form.                                          */
#define AP_JCOL_AUTO   0
#define AP_JCOL_DIRECT 1
#define AP_JCOL_FFT    2

typedef struct {
  int H, W;                  /* rows, columns (>= 1)                             */
  double A[4];               /* pixel->world matrix, row-major [[A0 A1][A2 A3]]; */
  double origin[2];          /* world position of pixel corner (0, 0)            */
  const float* data_dev;     /* H*W observed image                               */
  const float* variance_dev; /* H*W sigma^2 map (Sec. "chi^2 Optimization")       */
  const uint8_t* mask_dev;   /* H*W, 1 = excluded; NULL = no mask                 */
  const float* psf_dev;      /* K*K PSF image, NULL = no PSF; normalised to unit
                                sum by the library (Sec. "PSF convolution")       */
  int K;                     /* odd PSF size (ignored when psf_dev is NULL and
                                psf_live is 0)                                    */
  int group;                 /* independent fitting problem this image belongs to */
  int psf_live;              /* 1: the PSF is a live model (Sec. "PSF
                                convolution"), a circular Moffat of size K x K
                                whose n and Rd are theta[psf_pidx[k]] (or
                                psf_pfix[k] where psf_pidx[k] = -1), rendered
                                per evaluation with the context's quadrature
                                rule, its centre on the middle pixel, on the
                                image's pixel grid (A), normalised to unit sum;
                                psf_dev is then ignored.  chi^2, the gradient,
                                the Jacobian and the LM step include d/d(n, Rd);
                                share the indices with the image's Moffat stars
                                to fit one PSF for both.  0: psf_dev as given */
  int psf_pidx[2];           /* theta indices of the live PSF's n and Rd        */
  double psf_pfix[2];        /* values of fixed live-PSF slots                   */
} ap_image_desc;

typedef struct {
  int type;                  /* AP_SERSIC ... AP_SKY_PLANE                        */
  int image;                 /* index into the image array                        */
  int win[4];                /* x0, x1, y0, y1: half-open pixel window, the region
                                where the model is evaluated (Sec. "Automatic
                                Initialization"); clipped to the image           */
  int psf_convolve;          /* 1: sampled on window + PSF half width and
                                convolved; 0: added unconvolved                  */
  int pidx[8];               /* theta index per slot, -1 = fixed at pfix[k];
                                shared parameters repeat an index                */
  double pfix[8];            /* values of fixed slots                             */
} ap_source_desc;

/* Create a context bound to opt->device.  *out receives the handle. */
int ap_create(ap_ctx** out, const ap_options* opt);

/* Free every device and host resource of the context (NULL is a no-op). */
void ap_destroy(ap_ctx* ctx);

/* Static text of a status code. */
const char* ap_strerror(int code);

/* One-line description of the context's last failure ("" if none). */
const char* ap_get_error(ap_ctx* ctx);

/* Describe the problem (Sec. "Image Modeling" and "chi^2 Optimization"):
 * n_img images, n_src sources, a theta of n_params entries.  The descriptors
 * are copied; the image buffers they point to must stay valid until the next
 * ap_set_problem() or ap_destroy().  Builds the window / tile plans (the
 * structure is fixed for the whole fit), uploads them, normalises the PSFs and
 * allocates scratch.  Synchronises the stream.  Errors: AP_ERR_ARG for an
 * invalid descriptor (message names it), AP_ERR_NOMEM, AP_ERR_CUDA. */
int ap_set_problem(ap_ctx* ctx, const ap_image_desc* imgs, int n_img,
                   const ap_source_desc* srcs, int n_src, int n_params, void* stream);

/* Layout facts of the current problem: number of groups, and for each theta
 * index its group (param_group_host, n_params ints, -1 = unused index). */
int ap_get_layout(ap_ctx* ctx, int* n_groups, int* param_group_host);

/* Model images at theta (Eq. chi2's m(i, theta): the sum of all sources on the
 * image, galaxies convolved with the normalised PSF).  model_dev[i] receives
 * image i as H*W values of the context precision (float for AP_PREC_MIXED,
 * double for AP_PREC_F64); a NULL entry skips that image. */
int ap_render(ap_ctx* ctx, const double* theta_dev, void* const* model_dev, void* stream);

/* chi^2 per group (Eq. chi2 without the 1/2 and the constant:
 * sum over unmasked pixels of (d - m)^2 / sigma^2) into chi2_dev[n_groups];
 * if grad_dev is not NULL, d chi^2 / d theta into grad_dev[n_params] through the
 * adjoint (Sec. "Implementation with PyTorch": back-propagation of chi^2 to
 * every parameter at about the cost of the forward model). */
int ap_eval(ap_ctx* ctx, const double* theta_dev, double* chi2_dev, double* grad_dev, void* stream);

/* ---- adaptive pixel integration (Sec. "Pixel Integration") ----------------
 * The model sampled with the paper's two-stage scheme instead of the fixed
 * order-Q rule of the context: per source, on its sampling box, a midpoint
 * pass; a budget e = tol |F| / N (F the source's midpoint flux on the box, N
 * its pixel count); order-3 Gauss-Legendre on the pixels whose discrete
 * Laplacian of the midpoint values (second differences of the three nearest
 * pixels of each axis inside the box) exceeds 24 e; where orders 3 and 2
 * differ by more than e, the pixel split 5 x 5 with order 5 on each
 * sub-pixel; where the summed orders 5 and 4 differ by more than e, each
 * sub-pixel whose order-5 and order-4 values differ by more than e / 25 split
 * 5 x 5 again with order 7.
 * Skies are linear in position and keep their (exact) midpoint value.
 *
 * chi2_dev[n_groups] (nullable) receives chi^2 as in ap_eval(); model_dev
 * (nullable) the model images as in ap_render().  levels_dev (nullable,
 * device, n_samples bytes from ap_get_adaptive_layout()) receives each
 * sample's final level: 0 midpoint, 1 order 3, 2 split with order 5, 3 split
 * again.  counts_host (nullable, 5 int64) receives the number of samples
 * ending at each level and the number of sub-pixels split again; it
 * synchronises the stream.  tol >= 0 (0 sends every pixel with a non-zero
 * Laplacian to the deepest level; the paper's default is 0.01).  The gradient
 * and the LM iteration keep the fixed rule.  The first call allocates the
 * scheme's scratch (2 values + 13 bytes per sample).  A problem with an
 * AP_PSF_STAR source is refused (AP_ERR_ARG): the scheme covers the analytic
 * profiles.  Errors: AP_ERR_ARG
 * (negative or non-finite tol), AP_ERR_STATE, AP_ERR_NOMEM, AP_ERR_CUDA. */
int ap_eval_adaptive(ap_ctx* ctx, const double* theta_dev, double tol, double* chi2_dev, void* const* model_dev,
                     uint8_t* levels_dev, int64_t* counts_host, void* stream);

/* ---- pixel-centred sampling with an interpolated re-shift (Sec. "PSF
 * convolution") ------------------------------------------------------------
 * The model as the paper's convolution mode builds it: every convolved
 * profile source (Sersic, exponential, Gaussian, Moffat with psf_convolve
 * set) is sampled (order-Q rule of the context) with its centre moved to the
 * centre of the pixel that holds it, then moved back by its sub-pixel offset
 * (du, dv) in [-1/2, 1/2) of the image's pixel grid, with method
 * AP_SHIFT_LANCZOS3 (Lanczos kernel, 3 lobes, weights normalised to unit
 * sum) or AP_SHIFT_BILINEAR, on its sampling box (zero beyond it), before the
 * PSF convolution (the interpolation is a discrete convolution: shifting
 * before or after the PSF is the same).  Other sources as in ap_render().
 * chi2_dev[n_groups] (nullable) receives chi^2 as in ap_eval(), model_dev
 * (nullable) the model images as in ap_render().  The gradient and the LM
 * iteration sample at the true centre.  The first call allocates the mode's
 * scratch (2 values per box pixel of every shifted source) and synchronises.
 * Errors: AP_ERR_ARG (method), AP_ERR_STATE, AP_ERR_NOMEM, AP_ERR_CUDA. */
#define AP_SHIFT_LANCZOS3 1
#define AP_SHIFT_BILINEAR 2
int ap_eval_shifted(ap_ctx* ctx, const double* theta_dev, int method, double* chi2_dev, void* const* model_dev,
                    void* stream);

/* Sample layout of the adaptive scheme: the total sample count, and for each
 * source the index of its first sample (offsets_host[n_src], -1 for skies and
 * empty boxes).  A source's samples cover its sampling box row-major: its
 * clipped window, grown by the PSF half width (K-1)/2 for a convolved source
 * and clipped to the image grown by that much.  Builds the plan (allocating)
 * if no adaptive call has yet. */
int ap_get_adaptive_layout(ap_ctx* ctx, int64_t* n_samples, int64_t* offsets_host);

/* Levenberg-Marquardt normal equations at theta (Sec. "Optimization
 * methods"): J^T W r into jtwr_dev[n_params] and J^T W J into the context's
 * sparse matrix, where J = dm/dtheta and W = diag(1/sigma^2, 0 if masked).
 * ap_get_jtwj_structure()/ap_copy_jtwj() read the matrix out. */
int ap_normal_eq(ap_ctx* ctx, const double* theta_dev, double* jtwr_dev, void* stream);

/* Number of stored entries of J^T W J (compressed sparse rows over theta). */
int ap_get_jtwj_nnz(ap_ctx* ctx, int64_t* nnz);
/* Row pointers (n_params + 1) and column indices (nnz) into host arrays. */
int ap_get_jtwj_structure(ap_ctx* ctx, int64_t* row_ptr_host, int32_t* col_idx_host);
/* Values (nnz doubles) of the last ap_normal_eq() into values_dev. */
int ap_copy_jtwj(ap_ctx* ctx, double* values_dev, void* stream);

/* One damped solve per group from the last ap_normal_eq():
 * (J^T W J + lambda_g D) delta = J^T W r, D = diag(J^T W J) floored at
 * 1e-12 of its largest entry, in float64.  lambda_dev[n_groups] is read and,
 * when a factorisation fails, raised x10 (up to 8 times) in place.  Groups of
 * up to 64 parameters use a dense Cholesky, larger ones block-Jacobi
 * preconditioned conjugate gradients to a relative residual of 1e-12. */
int ap_lm_solve(ap_ctx* ctx, double* lambda_dev, double* delta_dev, void* stream);

/* n_iter full LM iterations on device, each group independent (Sec.
 * "Optimization methods"): chi^2 and normal equations at theta, damped solve,
 * trial = clamp(theta + delta) to the parameter box, chi^2 at the trial; a
 * group accepts iff its chi^2 strictly decreases (lambda / 9), otherwise keeps
 * theta (lambda * 11).  theta_dev and lambda_dev are updated in place,
 * chi2_dev[n_groups] receives the chi^2 at the final theta.  The iteration is
 * captured once in a CUDA graph and replayed.  If log_host is not NULL it
 * receives n_iter * n_groups records {chi2_before, chi2_trial, lambda_after,
 * accepted} (4 doubles each) and the call synchronises the stream.
 * The first iteration evaluates the model of every group at theta.  The
 * trial's source records and weighted residual go to buffers of their own;
 * a group that accepts takes them over as its current ones, a group that
 * rejects keeps its current ones, so later iterations find theta's weighted
 * residual and chi^2 in place and evaluate the model once, at the trial
 * point.  (The gradient, Jacobian and J^T W J at theta are rebuilt in every
 * iteration.) */
int ap_lm_iterate(ap_ctx* ctx, double* theta_dev, double* lambda_dev, double* chi2_dev, int n_iter,
                  double* log_host, void* stream);

/* n_iter more LM iterations of the fit that the last ap_lm_iterate() or
 * ap_lm_continue() left in the context, as if that call had been given n_iter
 * more iterations (theta's weighted residual and chi^2 are taken from the
 * context, not evaluated again).  theta_dev[n_params], lambda_dev[n_groups] and
 * chi2_dev[n_groups] are outputs only (any may be NULL): the state after the
 * iterations.  log_host as in ap_lm_iterate().  The images' data, variance
 * and mask must not have changed since that call; after changing them, start
 * again with ap_lm_iterate().  Evaluations in between (ap_eval, ap_render,
 * ap_normal_eq) are allowed: the next iteration then evaluates at theta.
 * Returns AP_ERR_STATE if no ap_lm_iterate() has run since ap_set_problem(). */
int ap_lm_continue(ap_ctx* ctx, double* theta_dev, double* lambda_dev, double* chi2_dev, int n_iter,
                   double* log_host, void* stream);

/* ---- damped solve without device allocation ------------------------------
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory -- code running while a CUDA graph is being
 * captured (cudaMalloc is not a stream operation and is refused during
 * capture), processes confined to a fixed, pre-reserved memory budget, and
 * plug-ins whose host application owns every device allocation.
 *
 * Solves (A + lambda D) delta = jtwr for one group given as an n x n
 * symmetric CSR matrix on the device (row_ptr_dev[n+1], col_idx_dev[nnz]
 * sorted per row, vals_dev[nnz]; entries repeated at one position add up, in
 * the diagonal as in the product), D = diag(A) floored at 1e-12 of its largest
 * entry, by Jacobi-preconditioned conjugate gradients in float64 to a
 * preconditioned residual of 1e-11; a breakdown multiplies *lambda_dev by 10
 * and retries (up to 8 times).  lambda_dev (1 double) is read and written;
 * delta_dev receives n doubles; status_dev (1 int) receives AP_OK,
 * AP_ERR_TIMEOUT (4000 iterations without convergence) or AP_ERR_NOT_SPD.
 * Returns AP_ERR_ARG for n outside 1..AP_NOALLOC_MAX_N or a NULL pointer,
 * AP_ERR_CUDA if the launch or the set-up fails.
 *
 * Scratch: a fixed array of AP_NOALLOC_SCRATCH_DOUBLES doubles (768 KiB)
 * in the library's device data, which every GPU that loads the library holds
 * until the process exits.  The call allocates nothing and calls no
 * allocating routine.  A call made outside a stream capture looks up the
 * array's device address on the current device (the first one on a device
 * also loads the library's module there) and remembers it; a call made while
 * its stream is being captured uses the remembered address, so make the first
 * call on each device before any stream capture (otherwise AP_ERR_CUDA).
 * AP_ERR_CUDA is the launch's own failure, not an error left by earlier work.
 * All calls share the array and it keeps the last call's
 * contents (the kernel initialises everything it reads), so calls that
 * overlap on the GPU -- on different streams, or from different threads --
 * race: serialise them. */
#define AP_NOALLOC_MAX_N 16384
#define AP_NOALLOC_SCRATCH_DOUBLES (6 * AP_NOALLOC_MAX_N)
int ap_lm_solve_noalloc(int n, const int64_t* row_ptr_dev, const int32_t* col_idx_dev, const double* vals_dev,
                        const double* jtwr_dev, double* lambda_dev, double* delta_dev, int* status_dev,
                        void* stream);

/* Device status word: AP_OK, or the first AP_ERR_* a kernel raised (non-finite
 * variance, failed factorisation).  Synchronises the stream, then clears it. */
int ap_get_status(ap_ctx* ctx, int* status_host, void* stream);

/* Fit state for checkpointing and diagnostics (theta and lambda are the
 * caller's buffers): the per-group chi^2 of the last LM iteration
 * (chi2_host[n_groups]), the number of LM iterations run so far, and the
 * conjugate-gradient iteration count of each group's last solve
 * (cg_iters_host[n_groups], 0 for groups solved by Cholesky).  Any pointer may
 * be NULL.  Synchronises the device. */
int ap_get_state(ap_ctx* ctx, double* chi2_host, int64_t* iterations_host, int* cg_iters_host);

/* Kernels one LM iteration launches (kernel nodes of the captured graph; 0
 * before the first ap_lm_iterate()) and kernels the last ap_eval() launched. */
int ap_get_launch_count(ap_ctx* ctx, int* per_lm_iteration, int* per_eval);

/* The Jacobian-column convolution mode in use after ap_set_problem()
 * (AP_JCOL_DIRECT or AP_JCOL_FFT), the milliseconds one launch of each took
 * when the problem was planned (-1 where not timed: the float64 form, or a PSF
 * beyond the FFT block sizes), and the FFT mode's work: its blocks of 64 x 64
 * and of 128 x 128 (one per source, free slot and output block).  Any pointer
 * may be NULL. */
int ap_get_jcol_mode(ap_ctx* ctx, int* mode, double* ms_direct, double* ms_fft, int* fft_blocks_64,
                     int* fft_blocks_128);

/* Correlation tile variants (the direct PSF correlations of the model, the
 * adjoint and the Jacobian columns; Sec. "PSF convolution").  variant
 * receives the one the context runs (-1 before ap_set_problem()), n_variants
 * their number; shape_host (nullable, 3 ints per variant) the output tile
 * width and height in pixels and the threads of a CTA; ms_host (nullable, one
 * per variant) the milliseconds of one forward + adjoint correlation the
 * autotuner measured in ap_set_problem() (-1 where not timed: a forced
 * variant, or one whose shared memory does not fit the PSF). */
int ap_get_conv_variant(ap_ctx* ctx, int* variant, int* n_variants, int* shape_host, double* ms_host);

/* ---- diagnostics ----------------------------------------------------------
 * Throughput of one arithmetic pipe on the current device, measured by a
 * probe kernel (independent dependency chains in every thread of a full
 * grid; one warm-up launch, one timed launch), for the roofline fractions of
 * the path's kernels: AP_PIPE_FMA32 float32 FMA (2 flops each), AP_PIPE_XU
 * the special-function unit (ex2 and lg2, one op each), AP_PIPE_FMA64
 * float64 FMA (2 flops each), AP_PIPE_MMA_TF32 the warp-level TF32 MMA
 * m16n8k8 (2 x 16 x 8 x 8 flops each).  iters (1 .. 2^24) scales the work;
 * ms receives the launch's duration, ops the operations it executed.
 * Allocates a small buffer (stream-ordered) and synchronises the stream.
 * The paper has no counterpart: this measures the hardware, not the method. */
#define AP_PIPE_FMA32    0
#define AP_PIPE_XU       1
#define AP_PIPE_FMA64    2
#define AP_PIPE_MMA_TF32 3
int ap_measure_pipe(int kind, int iters, double* ms, double* ops, void* stream);

/* Per-kernel CUDA-event timing.  With timing on (ap_set_timing(ctx, 1)) every
 * launch of ap_eval(), ap_normal_eq(), ap_lm_solve() and ap_lm_iterate() is
 * bracketed by events on the caller's stream (ap_lm_iterate() then runs its
 * launches directly instead of through the graph).  ap_get_timing()
 * synchronises those events and returns, per kernel name, the average
 * duration in milliseconds (ms_host) and the number of launches (counts_host,
 * nullable) since the previous ap_get_timing(); names are written as a
 * ';'-separated list into names_host (size bytes). */
int ap_set_timing(ap_ctx* ctx, int on);
int ap_get_timing(ap_ctx* ctx, char* names_host, int size, double* ms_host, int* counts_host, int max_kernels,
                  int* n_kernels);

#ifdef __cplusplus
}
#endif
#endif /* ASTROPHOT_GB300_H */
