/*
 * nlem.h - C ABI of libnlem.so: constrained Euclidean medians by EM-ADMM and Non-Local
 * Euclidean Medians (NLEM) denoising on NVIDIA GB300 (sm_103a).
 *
 * Method: K. N. Chaudhury and K. R. Ramakrishnan, "A new ADMM algorithm for the Euclidean
 * median and its application to robust patch regression", arXiv 1501.03879.
 *
 * Conventions shared by every call
 *   - Return value: 0 = OK, > 0 = warning, < 0 = error (NLEM_ERR_*).  On error no work has
 *     been queued; nlem_last_error() returns a message (thread-local).
 *   - Array arguments are caller-owned DEVICE pointers unless the name ends in _host.  The
 *     library never frees or retains them beyond the call's stream work.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*, NULL = legacy
 *     default stream); outputs are valid once that stream has reached the call's work.
 *   - The library owns only what lives inside an nlem_ctx (workspace, tuning cache, graphs).
 *   - No C++ exception crosses this boundary.  Every entry point is thread-compatible: use
 *     one nlem_ctx per host thread.
 */
#ifndef NLEM_H_
#define NLEM_H_

#ifdef __cplusplus
extern "C" {
#endif

#define NLEM_OK 0
#define NLEM_WARN_NOT_CONVERGED 1   /* reserved: per-problem convergence is in iters_used */
#define NLEM_ERR_INVALID (-1)       /* an argument is out of range */
#define NLEM_ERR_CUDA (-2)          /* a CUDA call failed (message says which) */
#define NLEM_ERR_OOM (-3)           /* workspace allocation failed */
#define NLEM_ERR_TIMEOUT (-4)       /* a bounded device wait ran out */
#define NLEM_ERR_UNSUPPORTED (-5)   /* size outside what the kernels handle */

#define NLEM_PREC_FP32 0            /* patch distances in FP32 on CUDA cores */
#define NLEM_PREC_BF16 1            /* cross terms <P_i,P_j> in BF16 on tensor cores, FP32 accumulate */

#define NLEM_INIT_WEIGHTED_MEAN 0   /* z0 = P_C(sum w_j P_j / sum w_j): the NLM patch (Sec. 3) */
#define NLEM_INIT_NOISY_PATCH 1     /* z0 = P_C(P_i): the noisy patch (Sec. 3) */

#define NLEM_SOLVER_ADMM 0          /* EM-ADMM, Algorithm 1 (Sec. 2) */
#define NLEM_SOLVER_IRLS 1          /* IRLS on the smooth surrogate of Eq. 2 (Sec. 1), the comparison
                                       method of Sec. 3 (nlem_denoise only) */
#define NLEM_SOLVER_FAST 2          /* accelerated EM-ADMM: Algorithm 1's steps with momentum and
                                       restart (see nlem_options.restart_every) */

#define NLEM_PENALTY_UNIFORM 0       /* one penalty mu = rho for every constraint x_k = z: Algorithm 1 */
#define NLEM_PENALTY_WEIGHTED 1      /* a penalty per constraint, mu_k = rho * w_k (see nlem_options) */

#define NLEM_LAYOUT_AUTO 0          /* nlem_denoise picks the problem-to-CTA layout */
#define NLEM_LAYOUT_PIXEL 1         /* one pixel's problem per CTA */
#define NLEM_LAYOUT_PAIR 2          /* two horizontally adjacent pixels per CTA, sharing the points
                                       of their overlapping windows (patch 7, window <= 21) */

typedef struct nlem_ctx nlem_ctx;

/* C = [lo, hi]^d, the box of Sec. 3 (e.g. [0, 255] for 8-bit grayscale). */
typedef struct {
  float lo, hi;
} nlem_box;

/* Options shared by the solver entry points.  Fill with nlem_options_default(). */
typedef struct {
  float tol;          /* > 0: stop when both relative residuals < tol (checked every
                         check_every iterations and at the cap); <= 0: run exactly `iters` */
  int check_every;    /* residual check period m >= 1 */
  int precision;      /* NLEM_PREC_FP32 or NLEM_PREC_BF16 (nlem_denoise only) */
  int init;           /* NLEM_INIT_* (nlem_denoise only; em_solve_batch uses x0) */
  int fp64_check;     /* != 0: also compute, in FP64 on the GPU, the objective of problem (1)
                         and its optimality residual at the returned point (see outputs) */
  int layout;         /* NLEM_LAYOUT_* (nlem_denoise only); PAIR where the pair kernel does not
                         apply (BF16 precision, other patch sizes, window > 21, IRLS) is -5 */
  int solver;         /* NLEM_SOLVER_* (default ADMM).  IRLS is taken by nlem_denoise and
                         nlem_denoise_host only; every other entry point returns -1 for it */
  float irls_eps;     /* epsilon of the surrogate (Eq. 2), >= 1e-30 (default 1e-6) */
  int penalty;        /* NLEM_PENALTY_* (default UNIFORM).  WEIGHTED solves problem (1) with the
                         ADMM steps of Algorithm 1 under a penalty mu_k = rho * w_k on each
                         constraint x_k = z of the splitting (Sec. 2; Sec. 4 leaves the penalty
                         choice open): every prox radius w_k / mu_k becomes 1 / rho, the z-update
                         becomes the projected w-weighted mean of x_k + y_k / mu_k, and the
                         stopping rule's residuals are taken in the w-weighted norm (each point's
                         terms times w_k, n replaced by sum_k w_k).  Compiled for em_solve_batch
                         (and em_solve, em_solve_batch_host) with d = 49 and for nlem_denoise,
                         nlem_denoise_host and nlem_denoise_ex with 7x7 patches on the one-pixel
                         layout; -5 elsewhere (-1 with IRLS) */
  int restart_every;  /* NLEM_SOLVER_FAST only, >= 0.  The accelerated solver (Sec. 4 names accelerated
                         ADMM as future work) is fast ADMM with restart (Goldstein, O'Donoghue, Setzer
                         and Baraniuk 2014): each step is one step of Algorithm 1 from an extrapolated
                         point (z^, y^), followed by c = rho * n * ||z - z^||^2, the z-part of their
                         combined residual (its y-part lies below what FP32 iterates resolve near
                         convergence).  restart_every = 0 (default):
                         if c < 0.999 * c_prev, alpha+ = (1 + sqrt(1 + 4 alpha^2)) / 2 and z^, y^ step
                         past the new iterate by (alpha - 1) / alpha+ times its change; otherwise
                         alpha = 1, z^ and y^ restart from the previous iterate and c_prev is divided
                         by 0.999.  restart_every = k >= 1: the fixed restart of O'Donoghue and Candes
                         (2015), restarting after every k-th step and taking the momentum otherwise.
                         Stopping rule and residuals as Algorithm 1's at each step's x, y, z, with the
                         step's own z-change z - z^ in place of z - z_prev (the same without
                         extrapolation).  Compiled for em_solve_batch (and em_solve_batch_host)
                         with d = 49 and n <= 448, and for nlem_denoise, nlem_denoise_host and
                         nlem_denoise_ex with 7x7 patches and windows of at most 448 points on the
                         one-pixel layout (AUTO takes it; PAIR is -5), and for nlem_denoise_batch
                         (5x5 and 7x7 patches); -5 elsewhere and with per-point penalties */
} nlem_options;

void nlem_options_default(nlem_options* opt);

/* Last error message of the calling thread ("" if none). */
const char* nlem_last_error(void);

/* Library version string. */
const char* nlem_version(void);

/* Create / destroy a context bound to CUDA device `device`.  The context owns the
 * workspace, the tile-shape tuning cache and captured CUDA graphs. */
int nlem_ctx_create(nlem_ctx** ctx, int device);
int nlem_ctx_destroy(nlem_ctx* ctx);

/*
 * em_solve - one constrained Euclidean median, problem (1) of Sec. 1:
 *     z* ~ argmin_{z in C} sum_k w_k ||z - a_k||_2,  C = [box.lo, box.hi]^d,
 * by Algorithm 1 (EM-ADMM, Sec. 2) with penalty mu = rho, y_k = 0 and z started at
 * P_C(weighted mean), run for exactly `iters` iterations.
 *   points  [n][d] float32, row-major (device)      weights [n] float32 >= 0 (device)
 *   x_out   [d] float32 (device)
 * Errors: -1 if n < 1, d < 1 or d > 148, rho <= 0 or not finite, iters < 0, lo > hi or not
 * finite.  Points or weights that are not finite, or negative weights, give x_out = NaN.
 * iters == 0 returns P_C(weighted mean).
 */
int em_solve(nlem_ctx* ctx, const float* points, const float* weights, int n, int d,
             nlem_box box, float rho, int iters, float* x_out, void* stream);

/*
 * em_solve_batch - B independent problems of the same (n, d), Algorithm 1 on each.
 *   points   [B][n][d] float32 (device)     weights [B][n] float32 (device)
 *   x0       [B][d] float32 start points (device) or NULL for P_C(weighted mean)
 *   opt      options (NULL = defaults: fixed iteration count)
 *   x_out    [B][d] float32 (device)
 *   iters_used [B] int32 or NULL: iterations run (-1 marks a problem with non-finite
 *            input or a negative weight; its x_out is NaN)
 *   residual [B] float32 or NULL: max(r_pri, r_dual) at the last check, where
 *            r_pri  = sqrt(sum_k ||x_k - z||^2) / max(sqrt(sum_k ||x_k||^2), sqrt(n)||z||)
 *            r_dual = sqrt(n) ||z - z_prev|| / sqrt(sum_k ||y_k / rho||^2)
 *            (scaled-form ADMM residuals of Boyd et al. 2011, as cited in Sec. 2)
 *   obj64 / kkt64 [B] double or NULL (only with opt->fp64_check): F(z) of problem (1) and
 *            the projected-gradient optimality residual ||z - P_C(z - g/sum w)||, both in FP64.
 * Errors as em_solve; -5 if n exceeds the largest problem the on-chip (register + shared
 * memory) kernels hold for this d: 896 points for d = 25 and 49, 448 for d = 81, and for other
 * d <= 28 / 60 / 120 / 148: 512 / 256 / 256 / 256.  B == 0 returns 0 at once (the buffers may then be NULL).
 */
int em_solve_batch(nlem_ctx* ctx, const float* points, const float* weights, long long B, int n,
                   int d, nlem_box box, float rho, int iters, const float* x0,
                   const nlem_options* opt, float* x_out, int* iters_used, float* residual,
                   double* obj64, double* kkt64, void* stream);

/* Constraint sets C beyond the box (Algorithm 1 needs only a closed convex C with a simple
 * projection, Sec. 2).  The arrays are caller-owned DEVICE arrays of d floats. */
#define NLEM_SET_COORD_BOXES 1      /* prod_q [lo[q], hi[q]] (lo[q] <= hi[q] required) */
#define NLEM_SET_BALL 2             /* {x : ||x - center||_2 <= radius} */

typedef struct {
  int kind;              /* NLEM_SET_* */
  const float* lo;       /* COORD_BOXES: lower bounds [d] */
  const float* hi;       /* COORD_BOXES: upper bounds [d] */
  const float* center;   /* BALL: centre [d] */
  float radius;          /* BALL: finite, >= 0 */
} nlem_set;

/*
 * em_solve_batch_set - em_solve_batch with C = *set: the z-update of Algorithm 1 and the start
 * (x0, or the weighted mean) are projected onto the set instead of the box.  The coordinate
 * boxes clamp each coordinate; the ball pulls a point outside it radially onto the sphere.
 *   points, weights, x0, x_out, iters_used, residual: as em_solve_batch.
 * Runs on the box kernels' shapes: d <= 148, n at most 896 (d = 49), 512 (other d <= 28) or 256.
 * Errors: as em_solve_batch; -1 also for a NULL set, an unknown kind, NULL set arrays, a radius
 * that is negative or not finite, or the IRLS solver; -5 for n above the capacity or the FP64
 * check (its optimality residual is the box's).  B == 0 returns 0 at once.
 */
int em_solve_batch_set(nlem_ctx* ctx, const float* points, const float* weights, long long B, int n, int d,
                       const nlem_set* set, float rho, int iters, const float* x0, const nlem_options* opt,
                       float* x_out, int* iters_used, float* residual, void* stream);

/*
 * em_solve_batch_host - em_solve_batch on HOST buffers, with the copies pipelined against the
 * solves.  The batch runs in chunks of `chunk` problems (0 = about 1 GiB of points per chunk).
 * Chunk k+1's inputs are copied to the device on a context-owned copy stream while chunk k is
 * solved on `stream`; each chunk's results are copied back on `stream` after its solve.  Two
 * device chunks are double-buffered in the context workspace.  Waits for completion.
 *   points_host [B][n][d], weights_host [B][n] float32 (host memory; pinned memory lets the
 *   copies overlap the solves, pageable memory works without overlap)
 *   x0_host [B][d] or NULL;  x_out_host [B][d];  iters_used_host [B] int32 or NULL;
 *   residual_host [B] float32 or NULL: as em_solve_batch.  The FP64 check outputs are not
 *   returned here (use em_solve_batch).
 * Errors as em_solve_batch; -1 also for chunk < 0; -3 if the chunk workspace cannot be allocated.
 * B == 0 returns 0 at once (the buffers may then be NULL), as em_solve_batch does.
 */
int em_solve_batch_host(nlem_ctx* ctx, const float* points_host, const float* weights_host, long long B,
                        int n, int d, nlem_box box, float rho, int iters, const float* x0_host,
                        const nlem_options* opt, long long chunk, float* x_out_host,
                        int* iters_used_host, float* residual_host, void* stream);

/*
 * nlem_denoise - NLEM of Sec. 3 (Eq. L1regression) on one grayscale image.
 * For every pixel i: P_j = the patch x patch window of the image centred at j
 * (reflect-padded at the border, no edge repeat), S(i) = centres j of the window x window
 * search window around i that lie in the image (clipped at the border, so n varies),
 * w_ij = exp(-||P_i - P_j||^2 / h^2) (not divided by patch^2; w_ii = 1), then EM-ADMM over
 * C = [box.lo, box.hi]^(patch^2) with mu = rho, and out[i] = centre coordinate of the solution.
 *   image [H][pitch] float32 (device), pitch >= W elements
 *   out   [H][W] float32 (device)
 *   iters_used [H][W] int32 or NULL;  residual [H][W] float32 or NULL (as em_solve_batch)
 *   obj64 / kkt64 [H][W] double or NULL (opt->fp64_check; weights recomputed in FP64)
 * opt->precision = NLEM_PREC_BF16: the cross terms <P_i, P_j> of the squared distances
 * ||P_i||^2 + ||P_j||^2 - 2 <P_i, P_j> are computed from bfloat16-rounded patches on the
 * tensor cores (tcgen05, FP32 accumulation), the norms in FP32, into a context-owned weight
 * table; the ADMM iterations stay in FP32.  Patch 5, 7 or 9.
 * opt->layout: PAIR runs the pixel-pair kernel (pixels (y, 2m) and (y, 2m+1) in one CTA,
 * every shared window point read once for both; patch 7, FP32, window <= 21); PIXEL one
 * pixel per CTA; AUTO takes PAIR for patch 7 in FP32 with window 17..21 and PIXEL otherwise.
 * Each pixel still stops at its own residual check, so the layouts differ only by FP32
 * rounding order.
 * opt->solver = NLEM_SOLVER_IRLS (NLEM-IRLS, the comparison method of Sec. 3): each pixel's
 * problem is solved by IRLS on the surrogate of Eq. 2 instead of EM-ADMM,
 *     x <- P_C(sum_k om_k a_k / sum_k om_k),  om_k = w_k (||x - a_k||^2 + irls_eps)^(-1/2),
 * from the same start point, for exactly `iters` steps (opt->tol must be <= 0; rho is not
 * used but must still be valid).  iters_used = iters; residual = ||x(T) - x(T-1)|| / ||x(T)||
 * of the last step; obj64 / kkt64 as for EM-ADMM (the objective of problem (1) at x(T)).
 * One pixel per CTA (layout PAIR is -5); patch 5, 7 or 9.
 * Errors: -1 if patch or window is even or < 1, patch > min(H, W),
 * h <= 0, rho <= 0, iters < 0, lo > hi; -5 if patch*patch > 128 or the window holds more
 * points than the kernels support (window <= 31).
 */
int nlem_denoise(nlem_ctx* ctx, const float* image, int H, int W, int pitch, int patch,
                 int window, float h, float rho, int iters, nlem_box box,
                 const nlem_options* opt, float* out, int* iters_used, float* residual,
                 double* obj64, double* kkt64, void* stream);

/*
 * nlem_denoise_color - NLEM of Sec. 3 on a multichannel image.  The patch of pixel j stacks the
 * channels' patch x patch patches (coordinate q = c*patch^2 + r*patch + s, d = channels*patch^2),
 * so ||P_i - P_j||^2 sums over all channels and C = [box.lo, box.hi]^d; otherwise as
 * nlem_denoise (reflect padding, clipped windows, weights, start, EM-ADMM, stopping rule).
 *   image [channels][H][pitch] float32 (device), channel planes H*pitch elements apart
 *   out   [channels][H][W] float32 (device): the centre coordinate of each channel
 *   iters_used, residual [H][W] or NULL; obj64 / kkt64 [H][W] or NULL (opt->fp64_check)
 * FP32 weights, EM-ADMM.  Compiled for 3 channels with patch 5 (d = 75, windows up to 21, one
 * pixel per CTA) and patch 7 (d = 147, windows up to 21).  With patch 7, windows of more than 256
 * points split each pixel over a cluster of two CTAs that add their partial sums every iteration
 * through distributed shared memory; the FP64 check is available up to 256 points (window 15).
 * Errors: as nlem_denoise; -5 for other channel counts or patches, larger windows, BF16
 * precision, the pair layout or the FP64 check on a split window; -1 for the IRLS solver.
 */
int nlem_denoise_color(nlem_ctx* ctx, const float* image, int H, int W, int pitch, int channels, int patch,
                       int window, float h, float rho, int iters, nlem_box box, const nlem_options* opt, float* out,
                       int* iters_used, float* residual, double* obj64, double* kkt64, void* stream);

/*
 * nlem_denoise_host - nlem_denoise on HOST buffers: copies image_host [H][W] to the device,
 * denoises, copies out_host [H][W] back, and waits for completion.  Uses context workspace.
 * Host buffers may be pageable or pinned (pinned is faster).
 */
int nlem_denoise_host(nlem_ctx* ctx, const float* image_host, int H, int W, int patch, int window,
                      float h, float rho, int iters, nlem_box box, const nlem_options* opt,
                      float* out_host, int* iters_used_host, void* stream);

/* One image of a batch.  The struct itself is host memory; its pointers are device pointers. */
typedef struct {
  const float* image;   /* [H][pitch] float32 */
  float* out;           /* [H][W] float32 */
  int* iters_used;      /* [H][W] int32 or NULL */
  float* residual;      /* [H][W] float32 or NULL */
  int H, W, pitch;
  int patch, window;    /* odd; patch 5 or 7 in the batched kernel; window^2 <= 441 */
  float h;              /* weight scale, e.g. 10 * sigma */
} nlem_image_desc;

/*
 * nlem_denoise_batch - NLEM (as nlem_denoise) on `count` images of uneven sizes, patch and
 * window sizes in ONE persistent kernel launch: every (image, pixel) pair is a work item that
 * CTAs take from a device work queue in the context workspace.  The queue reset and the launch
 * are captured once in a CUDA graph per distinct batch (same descriptors and parameters) and
 * replayed on later calls.  The launch shape (kernel shape pair, items per queue access, CTAs
 * per SM) is chosen by the context's autotuner the first time a workload class is seen
 * (keyed by SM count, patch set, largest window and stopping mode); that first call runs a few
 * timed trials on a sample of the batch and synchronizes `stream`.
 * rho, iters, box and opt apply to every image; opt->precision must be FP32 and
 * opt->fp64_check is ignored.  opt->solver may be NLEM_SOLVER_FAST: the accelerated solver (see
 * nlem_options.restart_every) on its own shapes, one CTA of 256 threads per SM (ctas_per_sm of
 * nlem_batch_force_config does not apply to it); IRLS is -1.
 * Errors: -1 on an invalid descriptor (as nlem_denoise), -5 for patch sizes other than 5 and 7
 * or windows whose point count exceeds the batched kernel, -3 if the workspace cannot grow.
 */
int nlem_denoise_batch(nlem_ctx* ctx, const nlem_image_desc* images, int count, float rho, int iters,
                       nlem_box box, const nlem_options* opt, void* stream);

/* Text description of the launch shape the last nlem_denoise_batch call used (NUL-terminated,
 * truncated to len).  Returns 0, or -1 if no batch has run. */
int nlem_batch_config(nlem_ctx* ctx, char* buf, int len);

/*
 * nlem_batch_force_config - pins the launch shape of the context's next nlem_denoise_batch calls
 * instead of the autotuner's choice (variant -1 restores the autotuner).  variant 0: one solver
 * shape per patch size (448 point slots for 7x7 patches, 512 for 5x5); variant 1: a shape per
 * window-size class (7x7: 128, 256 or 448 slots; 5x5: 256 or 512), so that small windows do not
 * iterate over empty slots.  fetch >= 1 work items per queue access, 1 or 2 CTAs per SM.  Drops the
 * captured graph.  Errors: -1 for a NULL ctx or values out of range.
 */
int nlem_batch_force_config(nlem_ctx* ctx, int variant, int fetch, int ctas_per_sm);

/*
 * nlem_denoise_batch_noalloc - nlem_denoise_batch for callers that cannot allocate device
 * memory: code that runs inside another framework's allocator or memory pool, or under a
 * memory budget in which every device allocation belongs to the host application, and so may
 * not call cudaMalloc (or anything that does) behind its back.  No paper counterpart: the
 * method itself needs no allocation; this entry point only moves the batched launch's scratch
 * (its work-queue counter and image descriptors) into a fixed array that the library holds.
 *   - Makes no device (or heap) allocation and needs no nlem_ctx; runs on the current device
 *     and `stream`; images and options as for nlem_denoise_batch (patch 5 or 7,
 *     window^2 <= 441; Algorithm 1, or the accelerated solver with opt->solver =
 *     NLEM_SOLVER_FAST and opt->restart_every).
 *   - At most NLEM_NOALLOC_MAX_IMAGES images per call (-1 above that).  The array
 *     (about 18 KB) stays resident on every GPU that loads the library until the process exits.
 *   - Each call looks up the array's device address in the current context
 *     (cudaGetSymbolAddress, which allocates nothing), so the address stays right after
 *     cudaDeviceReset or under a caller's own driver-API context.  The first call in a context
 *     also loads the library's device code there.
 *   - Every call shares the one array: the descriptors are rewritten and the counter is reset
 *     on each call, so calls whose GPU work overlaps (different streams, or different host
 *     threads, with no ordering between them) race and corrupt each other.  Order them.
 *   - Uses a fixed launch shape (no autotuning, no CUDA graph).
 * Errors as nlem_denoise_batch; messages via nlem_last_error().
 */
#define NLEM_NOALLOC_MAX_IMAGES 256
int nlem_denoise_batch_noalloc(const nlem_image_desc* images, int count, float rho, int iters,
                               nlem_box box, const nlem_options* opt, void* stream);

/*
 * nlem_bf16_weights - the weight stage of the mixed-precision path on its own: for every
 * pixel i and every centre j of its clipped search window, in NLEM's window order,
 *   wtab[i * window^2 + j] = exp(-(||P_i||^2 + ||P_j||^2 - 2 <bf16(P_i), bf16(P_j)>) / h^2)
 * (Sec. 3's weights with the cross term from bfloat16-rounded patches on the tensor cores,
 * FP32 accumulation; norms in FP32; negative squared distances from rounding become 0).
 * wtab: device [H*W][window^2] float32; entries j >= the pixel's window size are not written.
 * Patch 5, 7 or 9; window <= 31.  A bounded-wait timeout is reported by nlem_device_status.
 */
int nlem_bf16_weights(nlem_ctx* ctx, const float* image, int H, int W, int pitch, int patch,
                      int window, float h, float* wtab, void* stream);

/*
 * nlem_device_status - waits for the device and reports faults the kernels detected on their
 * own: NLEM_ERR_TIMEOUT if a bounded wait of the BF16 tensor-core weight kernel ran out (the
 * flag is then cleared), NLEM_ERR_CUDA for a CUDA error, 0 otherwise.
 */
int nlem_device_status(nlem_ctx* ctx);

/*
 * nlem_selftest_timeout - exercises the bounded-wait path on the device: runs the BF16 weight
 * kernel on a 16 x 16 image with its tensor-core step withheld and a 256-poll bound, so that
 * every CTA's wait runs out, flags the timeout, frees its TMEM and returns.  Returns what
 * nlem_device_status then reports: NLEM_ERR_TIMEOUT when the path works (the flag is cleared and
 * the context stays usable).  Synchronous.
 */
int nlem_selftest_timeout(nlem_ctx* ctx);

/* ------------------------------------------------------------------------------------------
 * Learned warm start (not in the paper, which starts from the noisy or the NLM patch and
 * uses one penalty mu for all problems): a 3-layer MLP with FP16 weights and FP32 arithmetic,
 * 2d+2 inputs -> 128 -> 128 -> d+1 outputs (ReLU between layers), maps a problem's features
 *   f = [m (d): weighted mean sum p_k a_k, q (d): coordinate-wise lower weighted median,
 *        H = -sum p_k ln p_k, pmax = max p_k],  p_k = w_k / sum w,
 * (inputs normalised as (v - 127.5)/64 for m and q, H / ln(nref), pmax as is) to
 *   x0 = P_C(m + 16 * y[0:d]),  rho = exp(clamp(y[d], -12, 4)).
 * Trained on solves the method itself produces (nlem_ws_labels gives the labels) with the
 * library's own forward, backward and Adam kernels.  Parameter vector layout (row-major):
 *   W1 [128][2d+2], b1 [128], W2 [128][128], b2 [128], W3 [d+1][128], b3 [d+1].
 * ------------------------------------------------------------------------------------------ */
typedef struct nlem_warmstart nlem_warmstart;

/* Number of parameters of the model for dimension d (-1 if d < 1). */
long long nlem_ws_num_params(int d);
/* New model for dimension d (1..81) with seeded He-normal weights on the context's device;
 * nref normalises the entropy input (use the largest window size n, e.g. 441). */
int nlem_ws_create(nlem_ctx* ctx, int d, float nref, unsigned long long seed, nlem_warmstart** ws);
int nlem_ws_destroy(nlem_warmstart* ws);
/* FP32 master parameters to / from host memory (set also resets the Adam state). */
int nlem_ws_get_params(nlem_warmstart* ws, float* host_params);
int nlem_ws_set_params(nlem_warmstart* ws, const float* host_params);
/* Binary checkpoint: "NLEMWS01", d, hidden, nref, Adam step, parameters, Adam moments. */
int nlem_ws_save(nlem_warmstart* ws, const char* path);
int nlem_ws_load(nlem_warmstart* ws, const char* path);
/* y [B][d+1] = network(feats [B][2d+2]) (device arrays). */
int nlem_ws_forward(nlem_ctx* ctx, nlem_warmstart* ws, const float* feats, long long B, float* y, void* stream);
/* Loss L = (1/B) sum_b [(1/d) sum_{c<d} (y_bc - t_bc)^2 + (y_bd - t_bd)^2] of a batch and its
 * gradient with respect to the FP32 parameters (forward with the FP16 weights).
 * loss: device float or NULL; grad: device [num_params] or NULL (kept inside ws). */
int nlem_ws_loss_grad(nlem_ctx* ctx, nlem_warmstart* ws, const float* feats, const float* targets, long long B,
                      float* loss, float* grad, void* stream);
/* One Adam step (lr, beta 0.9 / 0.999, eps 1e-8) on the loss of the batch. */
int nlem_ws_train_step(nlem_ctx* ctx, nlem_warmstart* ws, const float* feats, const float* targets, long long B,
                       float lr, float* loss, void* stream);
/* Training on a whole set: `epochs` passes over feats [N][2d+2] and targets [N][d+1] (device),
 * each in a fresh order (a Fisher-Yates shuffle drawn from SplitMix64 in counter mode under
 * `seed`), one nlem_ws_train_step per full minibatch of `batch` rows (min(batch, N); the
 * N mod batch rows an epoch leaves out come up in later epochs' orders).  epoch_loss: host
 * [epochs] or NULL, the mean minibatch loss of each epoch (reading it waits for the device).
 * The library owns the order and minibatch workspace inside ws.  Errors: -1 for N < 1,
 * epochs < 0, batch < 1 or lr not finite and > 0; -5 for N >= 2^31. */
int nlem_ws_train(nlem_ctx* ctx, nlem_warmstart* ws, const float* feats, const float* targets, long long N,
                  int epochs, int batch, float lr, unsigned long long seed, float* epoch_loss, void* stream);
/* y = network(feats), then x0 [B][d] and rho [B] as above (device arrays). */
int nlem_ws_predict(nlem_ctx* ctx, nlem_warmstart* ws, const float* feats, long long B, nlem_box box, float* y,
                    float* x0, float* rho, void* stream);

/* Features f (above) of the NLEM problems of the listed pixels (device linear indices, NULL =
 * all H*W in row-major order) into feats [npix or H*W][2d+2].  Patch 5, 7 or 9 and
 * (window + patch - 1)^2 <= 1024 (the pixel's tile is sorted in one 1024-entry sort); a listed
 * index outside [0, H*W) gives a row of NaN.  Errors: -1 as nlem_denoise, or npix < 0 with a
 * list; -5 otherwise unsupported. */
int nlem_features(nlem_ctx* ctx, const float* image, int H, int W, int pitch, int patch, int window, float h,
                  const int* pixels, long long npix, float* feats, void* stream);

/* nlem_denoise on the listed pixels only (NULL = all), optionally from per-pixel start points
 * x0 [pixel][d] and penalties rho_pix [pixel] (device, indexed by linear pixel), writing the
 * centre pixel to out[pixel] and optionally the whole solution patch to z_out [pixel][d].
 * A listed index outside [0, H*W) is skipped. */
int nlem_denoise_ex(nlem_ctx* ctx, const float* image, int H, int W, int pitch, int patch, int window, float h,
                    float rho, int iters, nlem_box box, const nlem_options* opt, const int* pixels, long long npix,
                    const float* x0, const float* rho_pix, float* out, int* iters_used, float* residual,
                    float* z_out, void* stream);

/* Training labels of the warm start for the listed pixels of one image (device linear indices,
 * n of them), from solves the method itself produces (Algorithm 1 on the pixels' Sec. 3 problems,
 * weighted-mean start, box C):
 *   rho* = the penalty of rho_grid (host, n_rho of 1..64) that reaches relative residual tol
 *          (checked every check_every iterations, cap `cap`) in the fewest iterations, the first
 *          in grid order on a tie;
 *   z*   = the solution patch of a tight solve (tight_tol, cap tight_cap) at rho*;
 *   targets [n][d+1] (device) = [(z* - m) / 16, ln rho*], m = feats[i][0:d] (feats [n][2d+2]:
 *          nlem_features of the same list).
 * rho_counts (host [n_rho], nullable): how many pixels each grid penalty won (the call then waits
 * for the device).  Entries outside [0, H*W) get NaN targets.  Workspace (about H*W*(d + 3)
 * floats) is held by the context.  Errors: -1 for bad arguments (as nlem_denoise, or NULL
 * arrays, a grid value that is not finite and > 0, tol or tight_tol not > 0, a cap < 1). */
int nlem_ws_labels(nlem_ctx* ctx, const float* image, int H, int W, int pitch, int patch, int window, float h,
                   nlem_box box, const int* pixels, long long n, const float* rho_grid, int n_rho, float tol,
                   int check_every, int cap, float tight_tol, int tight_cap, const float* feats, float* targets,
                   long long* rho_counts, void* stream);

/* NLEM with the learned warm start: features -> network -> EM-ADMM from (x0, rho) with the
 * stopping rule of opt (opt->tol > 0 required) and the cap iters; every pixel that reaches
 * the cap is solved again by plain EM-ADMM (weighted-mean start, penalty rho_fallback).
 * iters_used (required) holds the iterations of the solve that produced out.
 * fallback_count (host, nullable): if given, the call waits and reports how many pixels fell
 * back.  Workspace for the features and predictions is held by the context. */
int nlem_denoise_warm(nlem_ctx* ctx, nlem_warmstart* ws, const float* image, int H, int W, int pitch, int patch,
                      int window, float h, float rho_fallback, int iters, nlem_box box, const nlem_options* opt,
                      float* out, int* iters_used, long long* fallback_count, void* stream);

/*
 * nlem_debug_status - the bounds-check record of the debug build (libnlem_debug.so, built with
 * -DNLEM_DEBUG): every shared-memory tile, point-row and image index that depends on the image
 * size, window clipping, reflect padding or work-item lookup is checked against what it indexes;
 * an index outside it is recorded and the access skipped (a load reads 0).  Waits for the device,
 * then reports the first fault (site: the nlemk::DebugSite of csrc/debug.h, index, limit) and
 * the number of faults since the last reset (0 = none); reset != 0 clears the record.  A tool for
 * development (the sanitizer's stand-in), not part of the method.  Returns -5 in the release
 * build (no checks compiled; outputs 0).
 */
int nlem_debug_status(int reset, int* site, long long* index, long long* limit, long long* count);

/*
 * nlem_fp32_peak - measured FP32 FMA throughput of the current device (TFLOP/s, counting an
 * FMA as 2 flops), from a register-only FMA-chain kernel timed with CUDA events; also
 * returns the SM count.  Used as the roofline denominator of the ALU-bound kernels.
 */
int nlem_fp32_peak(nlem_ctx* ctx, double* tflops, int* sm_count);

#ifdef __cplusplus
}
#endif
#endif /* NLEM_H_ */
