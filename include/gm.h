/*
 * gm.h -- C ABI of libgm: batched galaxy-profile fitting on one B300 (sm_103a).
 *
 * The library evaluates, for a whole batch of galaxy stamps at once, the
 * forward model of arxiv 2404.07780 ("galmoss"): light profiles on the
 * elliptical radius (Sec. 4.1-4.2: Eqs. r, rmaj, rmin with B = 0, and
 * sersic-intensity, expdisk_I, ferrer_I, BE_S, gaussion_I, moffat_I, sky_I),
 * summed, correlated with each galaxy's PSF (Sec. 2 workflow, App. C conv2d
 * with padding="same"), plus the unconvolved components; the masked
 * sigma-weighted chi^2 (Sec. 5.1, Eq. chinu); the analytic Jacobian reduced to
 * per-galaxy J^T W J and J^T W r; and a batched Levenberg-Marquardt update
 * with the covariance uncertainty of Sec. 5.2.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Pointers.  Every array argument is a DEVICE pointer on the current CUDA
 *   device unless its comment says "host".  The caller owns all memory; the
 *   library allocates nothing.  Scratch memory is the caller's `workspace`,
 *   sized by the matching *_workspace_bytes() query and 256-byte aligned.
 * Stream.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  gm_model and gm_chi2_grad only enqueue work; their outputs are
 *   valid once the stream has synchronised.  gm_fit_batch synchronises the
 *   stream to poll convergence and returns when the fit has finished.  The
 *   first call on a device that sets up profiles also fills the device's
 *   table of Sersic nu_n nodes and synchronises its stream once; while the
 *   stream is being captured into a graph that step is skipped and the set-up
 *   solves nu_n directly (the same constants).
 * Layout.  Stamps are row-major, H rows x W columns; the pixel in row i,
 *   column j has centre x = j + 0.5, y = H - 0.5 - i (row 0 at the top, the
 *   grid of the App. C listing).  Stamps and PSFs may all have one size or
 *   differ per galaxy (gm_batch.geom).  The PSF is applied as a cross-correlation,
 *   M[i,j] = sum_ab P[a,b] I[i+a-c, j+b-c] with c = (K-1)/2 and I = 0 outside
 *   the stamp (torch conv2d semantics); K must be odd; the PSF is used as
 *   given (normalise it yourself).
 * Mask.  uint8, nonzero = pixel excluded (Omega = 0 in Eq. chinu); NULL means
 *   every pixel is used.
 * Parameters.  params is [n_gal][n_slots] FP64 in physical units: pixels and
 *   radians.  Each component reads its parameters from the slots listed in
 *   gm_component.slot, in this order (geometric subset first, Sec. 2):
 *     GM_SERSIC   x0 y0 q pa Ie Re n
 *     GM_EXPDISK  x0 y0 q pa I0 rs
 *     GM_FERRER   x0 y0 q pa I0 rout a b        (zero for r >= rout)
 *     GM_KING     x0 y0 q pa I0 rc rt alpha     (zero for r >= rt; bracket read
 *                                                 so that I(0) = I0)
 *     GM_GAUSSIAN x0 y0 q pa I0 fwhm            (fwhm = 2 sqrt(2 ln 2) sigma)
 *     GM_MOFFAT   x0 y0 q pa I0 fwhm n
 *     GM_SKY      Isky                          (flat, Eq. sky_I)
 *     GM_TILTED_SKY Isky kx ky                  (Isky + kx (x - W/2) + ky (y - H/2), the
 *                                                 tilted sky of Eq. new_sky_I, measured from
 *                                                 the stamp centre)
 *   The elliptical radius is r = sqrt(X^2 + (Y/q)^2), X = cos(pa) dx +
 *   sin(pa) dy, Y = -sin(pa) dx + cos(pa) dy, floored at 1e-4 px (the general
 *   form with boxiness: gm_model_desc.has_box).  Two
 *   components that list the same slot share that parameter.
 * Errors.  Every entry point returns GM_OK (0) or a negative GM_E_* code and
 *   never aborts; gm_last_error() returns a message for the calling thread's
 *   last failure.  Per-galaxy problems are not call failures: they are
 *   reported through status_out (GM_ST_*).
 * Arithmetic.  Images FP32; profiles, correlation and per-tile reductions
 *   FP32; per-galaxy sums, the Sersic constant nu_n, the Cholesky solve and
 *   the LM state FP64.
 */
#ifndef GM_H
#define GM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GM_MAX_COMP 8
#define GM_MAX_SLOTS 24   /* parameter slots of a model */
#define GM_MAX_FREE 16    /* of which fitted (is_free) */

/* return codes */
#define GM_OK 0
#define GM_E_INVAL (-1)        /* bad argument (null pointer, bad size, bad descriptor) */
#define GM_E_CUDA (-2)         /* a CUDA runtime call failed */
#define GM_E_NOMEM (-3)        /* workspace smaller than the *_workspace_bytes() query */
#define GM_E_UNSUPPORTED (-4)  /* valid request outside what the library handles */
#define GM_E_TIMEOUT (-5)      /* a kernel's bounded wait for a tile load ran out (the
                                  kernel stopped instead of hanging); returned by the
                                  calls that synchronise (gm_fit_batch, gm_fit_adam,
                                  gm_bootstrap).  The asynchronous calls (gm_model,
                                  gm_chi2_grad, gm_chi2_grad_noalloc, gm_grad_adjoint)
                                  return GM_OK and write NaN to every output element of
                                  the call instead (which galaxy lost a tile is not
                                  recorded) */

/* per-galaxy fit status (status_out) */
#define GM_ST_RUNNING 0
#define GM_ST_CONVERGED 1      /* chi^2 decrease < tol, step < xtol or GN decrement < gtol chi^2 */
#define GM_ST_MAX_ITER 2       /* max_iter model+Jacobian evaluations spent */
#define GM_ST_STALLED 3        /* lambda exceeded lambda_max without a chi^2 decrease */
#define GM_ST_SINGULAR 4       /* damped normal matrix not factorisable up to lambda_max */
#define GM_ST_NONFINITE 5      /* chi^2 not finite at the starting point */
#define GM_ST_BAD_INPUT 6      /* sigma <= 0 or a non-finite image/sigma on a used pixel */
#define GM_ST_NO_DOF 7         /* used pixels <= free parameters */

typedef enum {
  GM_SERSIC = 1,
  GM_EXPDISK = 2,
  GM_FERRER = 3,
  GM_KING = 4,
  GM_GAUSSIAN = 5,
  GM_MOFFAT = 6,
  GM_SKY = 7,
  GM_TILTED_SKY = 8
} gm_kind;

/* One light-profile component.  slot[k] is the parameter slot holding this
 * component's k-th parameter (order in the header comment).  convolve = 1
 * correlates the component with the PSF; 0 adds it after the PSF (the flat sky
 * of Sec. 2 is added after the convolution). */
typedef struct {
  int32_t kind;
  int32_t convolve;
  int32_t slot[8];
} gm_component;

/* The model: components, and per slot whether it is fitted (is_free), fitted
 * in log space (is_log: the LM works on ln p, for positive scale and
 * amplitude parameters) and its bounds [lo, hi] (physical units; every trial
 * point is clamped to them).  Host memory. */
typedef struct {
  int32_t n_comp;                    /* 1..GM_MAX_COMP */
  gm_component comp[GM_MAX_COMP];
  int32_t n_slots;                   /* 1..GM_MAX_SLOTS, at most GM_MAX_FREE of them free */
  uint8_t is_free[GM_MAX_SLOTS];
  uint8_t is_log[GM_MAX_SLOTS];
  double lo[GM_MAX_SLOTS];
  double hi[GM_MAX_SLOTS];
  /* Magnitudes instead of amplitudes (Sec. 4.1-4.2): when amp_is_mag[c] is 1, the
   * amplitude slot of component c (Ie or I0) holds a magnitude m, and the
   * amplitude is the one that gives the component the total flux
   * 10^(-0.4 (m - mag_zero[c])): Eqs. sersicLtot, expdiskI0, ferrerI0 and
   * moffatI0 with r_box = 1 (B = 0), and I0 = flux / (2 pi q sigma^2) for the
   * Gaussian.  Not available for King and the skies (GM_E_UNSUPPORTED); the
   * slot must not be fitted in log space. */
  uint8_t amp_is_mag[GM_MAX_COMP];
  double mag_zero[GM_MAX_COMP];
  /* Boxiness (Eqs. r-rmin): when has_box[c] is 1 the component's radius is
   * r = (|X|^(B+2) + |Y/q|^(B+2))^(1/(B+2)) with B in slot comp[c].slot[np], np the
   * profile's parameter count above (B = 0 is the ellipse; B > 0 boxy, B < 0
   * discy; the slot's lower bound must exceed -2), and a magnitude amplitude
   * carries r_box = pi (2+B) / (2 beta(1/(2+B), 1/(2+B))) (Eq. rbox).  Sersic,
   * exponential disk, Gaussian and Moffat only (GM_E_UNSUPPORTED otherwise). */
  uint8_t has_box[GM_MAX_COMP];
} gm_model_desc;

/* A batch of stamps.  The struct itself is host memory; image, sigma, mask
 * and psf are device memory, geom is host memory.
 *
 * Equal stamps (geom == NULL): every stamp is H x W, every PSF K x K; stamp g
 * starts at element g*H*W, its PSF at g*K*K.
 * Uneven stamps (geom != NULL): geom[3g .. 3g+2] = (h_g, w_g, k_g) gives
 * galaxy g's stamp rows and columns (1..4096) and odd PSF side (1..63); H, W
 * and K are not read.  Stamps are packed back to back in galaxy order (stamp g
 * starts at sum_{g'<g} h_g' w_g'), PSFs likewise (sum_{g'<g} k_g'^2), and every
 * per-pixel output (model, components) follows the same packing.  The calls
 * read geom before they return and copy the derived tables to the workspace
 * with cudaMemcpyAsync from pageable memory, which may synchronise the stream. */
typedef struct {
  int32_t n_gal;            /* galaxies, >= 0 */
  int32_t H, W;             /* stamp rows, columns (1..4096); equal stamps only */
  int32_t K;                /* PSF side, odd, 1..63; equal stamps only */
  const float *image;       /* data D, [n_gal][H][W] or packed */
  const float *sigma;       /* uncertainty sigma (> 0 on used pixels), same layout */
  const uint8_t *mask;      /* same layout, or NULL */
  const float *psf;         /* [n_gal][K][K] or packed */
  const int32_t *geom;      /* NULL, or host [n_gal][3] = (h, w, k) of each galaxy */
} gm_batch;

/* Levenberg-Marquardt controls (host memory). */
typedef struct {
  double tol;          /* CONVERGED when an accepted step lowers chi^2 by < tol relative */
  double xtol;         /* CONVERGED when every internal step |du| <= xtol (|u| + xtol) */
  double gtol;         /* CONVERGED when the Gauss-Newton decrement g^T A^-1 g at the best
                          point is <= gtol chi^2 (checked at the start and after each accept) */
  int32_t max_iter;    /* model+Jacobian evaluations per galaxy (the start counts as one) */
  double lambda0;      /* initial damping */
  double lambda_up;    /* lambda *= lambda_up on a rejected step or a failed factorisation */
  double lambda_down;  /* lambda *= lambda_down on an accepted step ... */
  double lambda_min;   /* ... but not below lambda_min */
  double lambda_max;   /* STALLED / SINGULAR beyond this */
  int32_t polish;      /* 1: a CONVERGED fit takes one final Gauss-Newton step (gm_fit_batch); 0: none */
  int32_t canonical;   /* 1: at exit q > 1 is rewritten and position angles wrapped (gm_fit_batch);
                          0: params_out is the best point exactly as the fit holds it (a checkpoint) */
  double *lambda_inout;  /* NULL, or DEVICE [n_gal] FP64: each galaxy's starting damping (used
                            instead of lambda0 when > 0 and finite) in, its damping at exit out */
} gm_fit_opts;

/* Library version (major*10000 + minor*100 + patch). */
int gm_version(void);

/* Message for the calling thread's last nonzero return (static storage, never NULL). */
const char *gm_last_error(void);

/*
 * gm_model -- forward model of every galaxy (Sec. 2 workflow, Sec. 4 profiles).
 *   params     [n_gal][n_slots] FP64
 *   model_out  [n_gal][H][W] FP32: PSF-correlated sum of the convolved
 *              components plus the unconvolved ones
 *   comp_out   NULL or [n_gal][n_comp][H][W] FP32: each component's own
 *              contribution (correlated when the component is convolved);
 *              the stored image blocks of Sec. 2
 *   workspace  gm_model_workspace_bytes(desc, batch) bytes
 * Returns GM_E_INVAL for bad arguments, GM_E_NOMEM for a short workspace,
 * GM_E_UNSUPPORTED when K is too large for the tile to fit in shared memory.
 */
size_t gm_model_workspace_bytes(const gm_model_desc *desc, const gm_batch *batch);
int gm_model(const gm_model_desc *desc, const gm_batch *batch, const double *params,
             float *model_out, float *comp_out, void *workspace, size_t ws_bytes, void *stream);

/*
 * gm_chi2_grad -- chi^2 of Eq. chinu and its derivatives for every galaxy.
 *   params  [n_gal][n_slots] FP64
 *   chi2    [n_gal] FP64
 *   grad    NULL or [n_gal][n_slots] FP64: d chi^2 / d p in physical units,
 *           = -2 (J^T W r) with r = D - M and W = Omega / sigma^2; 0 for fixed slots
 *   jtj     NULL or [n_gal][n_slots][n_slots] FP64: J^T W J in physical units
 *           (the Gauss-Newton half-Hessian); rows/columns of fixed slots are 0
 *   workspace  gm_chi2_grad_workspace_bytes(desc, batch) bytes
 * The Jacobian is analytic (chain rule through the elliptical radius and each
 * profile), correlated with the PSF like the model.  A sigma <= 0 on a used
 * pixel gives a non-finite chi2 for that galaxy.
 */
size_t gm_chi2_grad_workspace_bytes(const gm_model_desc *desc, const gm_batch *batch);
int gm_chi2_grad(const gm_model_desc *desc, const gm_batch *batch, const double *params,
                 double *chi2, double *grad, double *jtj, void *workspace, size_t ws_bytes,
                 void *stream);

/*
 * gm_grad_adjoint -- chi^2 of Eq. chinu and d chi^2/dp by the adjoint of the
 * PSF correlation: with v = P^T (w r) (the same-size zero-padded correlation
 * with the PSF flipped in both axes),
 *   d chi^2/dp = -2 [ sum_pix (dI_conv/dp) v + sum_pix w r dI_unconv/dp ],
 * so a pass costs two single-channel correlations whatever the number of free
 * parameters (gm_chi2_grad correlates 1 + P channels and also returns
 * J^T W J).  The paper fits by gradient descent on this gradient (Sec. 5.1,
 * torch autograd); this is that gradient computed by hand.
 *   params  [n_gal][n_slots] FP64
 *   chi2    [n_gal] FP64
 *   grad    NULL or [n_gal][n_slots] FP64, physical units, 0 for fixed slots
 *   workspace  gm_grad_adjoint_workspace_bytes(desc, batch) bytes
 * Asynchronous on `stream` like gm_chi2_grad.  Equal stamps only: a batch with
 * geom returns GM_E_UNSUPPORTED (and the size query 0).  GM_E_INVAL for an even
 * or out-of-range PSF side, GM_E_NOMEM for a short or NULL workspace; an empty
 * batch (n_gal = 0) returns GM_OK without device work.
 */
size_t gm_grad_adjoint_workspace_bytes(const gm_model_desc *desc, const gm_batch *batch);
int gm_grad_adjoint(const gm_model_desc *desc, const gm_batch *batch, const double *params, double *chi2,
                    double *grad, void *workspace, size_t ws_bytes, void *stream);

/* Device time of each kernel group of one gm_grad_adjoint call (host memory).  Not
 * part of the paper's method: it lets a caller relate throughput to the kernels'
 * own time (the correlations are bound by the FP32 FMA pipe, the rest by issue). */
typedef struct {
  double setup_ms;     /* per-galaxy constants and the convolved profiles' pair planes */
  double resid_ms;     /* correlation of the profile planes with the PSFs (model) */
  double residual_ms;  /* residuals, chi^2 and the unconvolved components' terms */
  double grad_ms;      /* correlation of w r with the flipped PSFs (the adjoint) */
  double deriv_ms;     /* the convolved profiles' derivative sums and the per-galaxy totals */
} gm_adjoint_stats;

/* Kernel times of the calling thread's last gm_grad_adjoint (CUDA events recorded on
 * its stream; waits for that call to finish).  GM_E_INVAL if out is NULL or no call
 * has been timed on this thread (calls made while their stream was being captured
 * into a CUDA graph are not timed). */
int gm_grad_adjoint_last_stats(gm_adjoint_stats *out);

/*
 * gm_chi2_grad_noalloc -- gm_chi2_grad for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a convenience of the library.
 *
 * Who needs it: code that must not call cudaMalloc (or torch's allocator) at
 * the point where it evaluates chi^2 -- for example an optimiser or sampler
 * plugged into a host framework that owns every device buffer and only lends
 * it input and output pointers, or a pipeline stage that forbids allocation
 * after start-up because cudaMalloc can synchronise the device and fragment
 * memory.  Such callers still pass their inputs and outputs exactly as for
 * gm_chi2_grad (same arguments, same results); only the workspace is gone.
 *
 * Scratch: a fixed array of GM_NOALLOC_SCRATCH_BYTES inside the library,
 * reserved on every GPU that loads the library and held until the process
 * exits.  A request whose gm_chi2_grad_workspace_bytes() exceeds it returns
 * GM_E_NOMEM with a message (use gm_chi2_grad with your own workspace then).
 * Arguments are checked as by gm_chi2_grad, with the same messages (a bad
 * geometry of an uneven batch names the galaxy and the reason); an empty batch
 * (n_gal = 0) returns GM_OK without touching the device.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  Every
 * call shares the one array: calls that overlap on the GPU (two streams, or
 * two host threads) race and corrupt each other's results, so serialise them.
 * Nothing in the array carries over between calls (every call writes the
 * parts it reads).  The function calls no cudaMalloc, cudaFree or other
 * allocating routine.
 */
#define GM_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
int gm_chi2_grad_noalloc(const gm_model_desc *desc, const gm_batch *batch, const double *params,
                         double *chi2, double *grad, double *jtj, void *stream);

/*
 * gm_test_starve_next_pass -- a test of the timeout path; not part of the
 * paper's method.  Arms a one-shot fault on the host: the next tile-kernel
 * launch made by the calling thread (the fused pass of gm_model, gm_chi2_grad,
 * gm_chi2_grad_noalloc and the first iteration of gm_fit_batch, or the first
 * adjoint pass of gm_grad_adjoint and gm_fit_adam) has its first block skip the
 * load of its first window, so that its bounded wait finds nothing arriving and
 * gives up after `polls` polls instead of the normal limit, with no copy in
 * flight.  The call then reports the timeout as any other would (GM_E_TIMEOUT,
 * or NaN outputs; see GM_E_TIMEOUT).  polls = 0 disarms.  Always GM_OK.
 */
int gm_test_starve_next_pass(uint32_t polls);

/*
 * gm_fit_batch -- Levenberg-Marquardt fit of every galaxy (damped Gauss-Newton
 * on Eq. chinu; Sec. 5.1 names LM as the classical alternative to gradient
 * descent), with the covariance uncertainty of Sec. 5.2.
 *   params_inout [n_gal][n_slots] FP64: starting point in, best fit out
 *                (position angles wrapped to [0, pi)).  An axis ratio may
 *                exceed 1 during the fit (the same ellipse turned by pi/2);
 *                at exit q > 1 is rewritten as 1/q with the component's
 *                position angle + pi/2 and its scale lengths (r_e, r_s, r_out,
 *                r_c, r_t, fwhm) times q, which leaves the image unchanged,
 *                when those slots are not shared with components of another q
 *   opts         host; NULL = defaults (tol 1e-6, xtol 1e-10, gtol 1e-10, max_iter 100,
 *                lambda0 0.1, up 10, down 0.2, min 1e-7, max 1e10, polish 1, canonical 1,
 *                lambda_inout NULL)
 *   chi2_out     [n_gal] FP64 chi^2 at the best point
 *   dof_out      [n_gal] int32: used pixels - free parameters (Sec. 5.1)
 *   iters_out    [n_gal] int32: model+Jacobian evaluations spent
 *   status_out   [n_gal] int32: GM_ST_*
 *   sigma_p_out  NULL or [n_gal][n_slots] FP64: sqrt(diag (J^T W J)^-1) at the
 *                best point, in physical units (p * sigma_ln p for log slots);
 *                0 for fixed slots
 *   workspace    gm_fit_workspace_bytes(desc, batch) bytes
 * Each iteration: one model+Jacobian+reduction pass over the galaxies still
 * running, then one LM step per galaxy: solve (A + lambda diag A) delta = g
 * by FP64 Cholesky (A = J^T W J, g = J^T W r in internal coordinates: ln p
 * for log slots), trial = clamp(p + delta), accept if chi^2 drops.
 * Final Gauss-Newton step (opts->polish = 1): a fit that reaches CONVERGED
 * with evaluations to spare takes one undamped step delta = A^-1 g from its
 * best point (diag A floored at 1e-12 max diag A), evaluated in one more
 * iteration; its point becomes the result unless its chi^2 is non-finite or
 * above the best by more than 1e-6 relative.  The acceptance test above
 * compares chi^2 values accumulated from FP32 pixels, whose rounding (~1e-8
 * relative) exceeds what the last steps towards the minimum gain (~1e-10),
 * so that test alone can stop a fit short of the minimum; the final step is
 * taken from the gradient, whose FP32 error moves the minimum by ~1e-3 of the
 * parameters' 1e-4 relative tolerance.
 * Synchronises `stream` every few iterations to poll how many galaxies are
 * still running; returns when none is or all have spent max_iter.
 * Checkpoint and resume: a fit stopped at max_iter = k with canonical = 0 and
 * lambda_inout returns each galaxy's best point and damping as the fit holds
 * them; calling again from those (same lambda_inout) continues exactly: the
 * first evaluation reproduces the best point's normal equations bit for bit
 * (fixed-order sums), so every later step is the one the uninterrupted fit
 * takes.  For a galaxy still running at k, the resumed call with max_iter
 * N - k + 1 ends with the uninterrupted N-iteration fit's results, bit for
 * bit, its iters_out being one more than the remaining evaluations (the
 * best point is evaluated again).  Galaxies that finished before k are
 * resumed as new fits: pass only the ones still running.
 */
size_t gm_fit_workspace_bytes(const gm_model_desc *desc, const gm_batch *batch);

/* Counters of one gm_fit_batch call (host memory). */
typedef struct {
  int32_t passes;        /* fused model+Jacobian+reduction passes launched */
  int32_t graph_reused;  /* 1: the call replayed one of the thread's two most recent fit graphs (every
                            launch argument equal: same model, options, batch buffers, workspace); 0: it
                            recorded one */
  int64_t galaxy_evals;  /* galaxies evaluated, summed over the passes */
  int64_t converged;     /* galaxies that ended GM_ST_CONVERGED */
  int64_t iters_sum;     /* iters_out summed over the galaxies */
  double profile_ms;     /* device time of the profile kernels (channel images of each pass) */
  double fused_ms;       /* device time of the fused tile kernels (correlation + reduction) */
  double step_ms;        /* device time of the per-galaxy LM steps */
  double wall_ms;        /* host wall time of the call */
} gm_fit_stats;

/* Counters of the calling thread's last successful gm_fit_batch; GM_E_INVAL if
 * there was none or out is NULL.  Not part of the paper's method: it lets a
 * caller relate throughput to the kernels' own time. */
int gm_fit_last_stats(gm_fit_stats *out);

int gm_fit_batch(const gm_model_desc *desc, const gm_batch *batch, double *params_inout,
                 const gm_fit_opts *opts, double *chi2_out, int32_t *dof_out, int32_t *iters_out,
                 int32_t *status_out, double *sigma_p_out, void *workspace, size_t ws_bytes,
                 void *stream);

/*
 * gm_fit_adam -- the paper's own way of fitting (Sec. 5.1: gradient descent
 * embedded in torch, Sec. 2 workflow; its examples run 1,000 iterations): Adam
 * steps on chi^2 with the adjoint gradient of gm_grad_adjoint, for a fixed
 * number of iterations, all galaxies at once.  Equal stamps only.
 *   params_inout [n_gal][n_slots] FP64: the start in, the lowest-chi^2 point
 *                evaluated out (in canonical form, as gm_fit_batch returns it)
 *   chi2_out     [n_gal] FP64: chi^2 at that point
 *   workspace    gm_fit_adam_workspace_bytes(desc, batch) bytes
 * Steps are taken in internal coordinates (ln p for log slots, p otherwise)
 * and clamped to the bounds; the step of a linear slot is scaled by
 * max(|p at the start|, 1), so lr is a relative step for every slot.
 * Synchronises the stream once at the end.  The paper gives no learning rate
 * or moments for its optimiser: they are the caller's choice here.
 * GM_E_INVAL for NULL opts or n_iter < 1, lr <= 0, beta1 or beta2 outside
 * [0, 1), eps <= 0; GM_E_NOMEM for a short workspace.
 */
typedef struct {
  int32_t n_iter;   /* gradient evaluations followed by a step */
  double lr;        /* step size (relative, see above) */
  double beta1;     /* first-moment decay, e.g. 0.9 */
  double beta2;     /* second-moment decay, e.g. 0.999 */
  double eps;       /* e.g. 1e-8 */
} gm_adam_opts;

size_t gm_fit_adam_workspace_bytes(const gm_model_desc *desc, const gm_batch *batch);
int gm_fit_adam(const gm_model_desc *desc, const gm_batch *batch, double *params_inout, const gm_adam_opts *opts,
                double *chi2_out, void *workspace, size_t ws_bytes, void *stream);

/*
 * Bootstrap uncertainties (Sec. 5.2): every stamp's unmasked pixels are
 * resampled with replacement -- as many draws as there are such pixels --
 * and the galaxy is refitted from params_best; after n_boot replicates
 *   sigma_boot[g][s] = sqrt((1/M) sum_i (p_i - mean)^2)
 * over the M replicates whose refit CONVERGED (n_ok[g] = M; NaN when M = 0).
 * Position angles are taken within pi/2 of the best fit's.  A pixel drawn c
 * times enters chi^2 with weight c (sigma / sqrt(c)); undrawn pixels are
 * masked.  The draws come from SplitMix64 (Steele, Lea & Flood 2014) as a
 * counter-based generator: draw k of replicate b for galaxy g is the (k+1)-th
 * output of the SplitMix64 stream starting at the state
 * splitmix64(splitmix64(seed) ^ (g << 32 | b)), mapped to the pixel
 * floor(r N / 2^64) of the galaxy's N unmasked pixels in row-major order.
 * gm_bootstrap_counts writes the multiplicities of one replicate
 * ([n_gal][H][W] uint32) without fitting.  Equal stamps only; opts as
 * gm_fit_batch (NULL = defaults).  params_best, sigma_boot [n_gal][n_slots]
 * FP64, n_ok [n_gal] int32 (may be NULL).  Synchronises the stream (inside
 * each refit).  GM_E_INVAL for n_boot < 1, replicate < 0 or a NULL
 * params_best, sigma_boot or counts; GM_E_NOMEM for a short workspace.
 */
size_t gm_bootstrap_workspace_bytes(const gm_model_desc *desc, const gm_batch *batch);
int gm_bootstrap_counts(const gm_model_desc *desc, const gm_batch *batch, uint64_t seed, int32_t replicate,
                        uint32_t *counts, void *workspace, size_t ws_bytes, void *stream);
int gm_bootstrap(const gm_model_desc *desc, const gm_batch *batch, const double *params_best, int32_t n_boot,
                 uint64_t seed, const gm_fit_opts *opts, double *sigma_boot, int32_t *n_ok, void *workspace,
                 size_t ws_bytes, void *stream);

/*
 * Launch-shape tuning of the fused model+Jacobian pass (not part of the
 * paper's method: the hook of the autotuner in paper_2404_07780_b300/tune.py).
 *
 * gm_tune_set makes every later NORMAL-mode pass (gm_chi2_grad, gm_fit_batch,
 * gm_chi2_grad_noalloc) whose largest PSF side is K and that fits P free
 * parameters use this launch shape:
 *   pairs_per_pass    channel pairs loaded and correlated per shared-memory pass, 1..4
 *   pairs_per_thread  1 or 2
 *   groups            groups of 128 threads, 1..4 (1..2 with 2 pairs per thread,
 *                     or 4 with 2 pairs per thread and 4 or 2 pairs per pass:
 *                     each two (four) groups then split two pairs by PSF rows);
 *                     pairs_per_pass <= pairs_per_thread * groups
 * pairs_per_pass = 0 removes the (K, P) entry.  A shape that the device's
 * shared memory or the built kernels cannot run is ignored at launch in favour
 * of the default shape.  Results agree between shapes to FP32 rounding of the
 * per-tile sums.  The table is process-wide; gm_tune_clear empties it.
 * gm_tune_last_shape reports the shape of the calling thread's last planned
 * pass.  Returns GM_OK, or GM_E_INVAL for arguments outside these ranges.
 */
int gm_tune_set(int32_t K, int32_t P, int32_t pairs_per_pass, int32_t pairs_per_thread, int32_t groups);
int gm_tune_clear(void);
int gm_tune_last_shape(int32_t *pairs_per_pass, int32_t *pairs_per_thread, int32_t *groups);

#ifdef __cplusplus
}
#endif

#endif /* GM_H */
