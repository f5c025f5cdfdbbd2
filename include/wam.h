/*
 * libwam: multiresolution (wavelet-tree) alternating minimisation for
 * transmission CT on one GPU (sm_103a).
 *
 * Method: Degirmenci, O'Sullivan, Politte, "Multiresolution approach to
 * acceleration of iterative image reconstruction for X-ray imaging for
 * security applications" (arXiv 1508.04458).  Sec. II poses the problem:
 * counts d(y) with mean q(mu)(y) = I0(y) exp(-sum_x h(y|x) mu(x)), h(y|x)
 * the length of ray y inside voxel x, mu = Omega beta (Eq. 1.2) with Omega an
 * orthonormal Haar synthesis, minimised in I-divergence by Algorithm 1 over a
 * tree of active coefficients that grows as in the Results section.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Image: nx * ny pixels of vx * vy mm centred at the origin, row-major,
 *    x fastest: pixel (ix, iy) is mu[iy * nx + ix] and covers
 *    [-nx vx/2 + ix vx, ... + vx) x [-ny vy/2 + iy vy, ... + vy).
 *  - Scan: view k at theta_k = angle0 + k * angle_span / n_views,
 *    e = (cos, sin), u = (-sin, cos); bin b at
 *    u_b = (b - (n_bins - 1) / 2) * bin_pitch along u.  Parallel beam: ray =
 *    line through u_b u with direction e.  Flat-detector fan beam: ray = segment
 *    from the source SOD e to the detector point -(SDD - SOD) e + u_b u.
 *    Sinograms are [n_views][n_bins], ray index y = k * n_bins + b.
 *  - Haar coefficients (orthonormal, levels 1..L, block of a level-l
 *    coefficient = 2^l x 2^l pixels, basis value +-2^-l): vector of length
 *    nx*ny holding the level-L approximations ((ny>>L) x (nx>>L), row-major),
 *    then for l = L, L-1, ..., 1 the detail planes h_l, v_l, d_l (each
 *    (ny>>l) x (nx>>l)).  h is + on the lower-y half of its block, v is + on
 *    the lower-x half, d is their product.
 *  - Tree masks ("masks"): bytes, one per block and level, for l = L, L-1,
 *    ..., 1 in turn, each level (ny>>l) x (nx>>l) row-major; nonzero = the
 *    block is expanded, i.e. its three level-l details are active.  The
 *    level-L approximations are always active.  Total size wam_mask_bytes().
 *  - Cone beam (kind WAM_CONE3D_FLAT_CIRCULAR): volume nx*ny*nz voxels,
 *    index (iz*ny + iy)*nx + ix, centred at the origin; ray (view k, row r,
 *    bin b) from the source SOD e (z = 0) to -(SDD - SOD) e + u_b u + v_r z,
 *    v_r = (r - (n_rows - 1)/2) * row_pitch; sinogram [n_views][n_rows][n_bins].
 *    Two wavelet modes (wam_schedule.dims): 3 = orthonormal 3-D Haar (block of
 *    2^l voxels per side, value +-2^(-3l/2); seven details of type t = 1..7,
 *    a bit mask of the differenced axes x = 1, y = 2, z = 4, - on the upper
 *    half; layout: level-L approximations z-major, then for l = L..1 the planes
 *    t = 1..7, each (nz>>l, ny>>l, nx>>l); masks per level (nz>>l)(ny>>l)(nx>>l));
 *    2 with zsum_criterion = 1 = the 2-D Haar above applied to every z-slice
 *    (coefficients slice-major, nx*ny per slice) under one 2-D tree shared
 *    by all slices, expansion criterion S = sum over z of mu.  Cone-beam
 *    contexts support wam_set_data, wam_reconstruct (precision 32),
 *    wam_project, wam_backproject and the measurement calls; the other
 *    step-level calls return WAM_ERR_ARG.
 *  - Pointers named on_device / documented as device pointers are
 *    caller-owned CUDA device memory used on `stream` (a cudaStream_t, NULL =
 *    the legacy default stream); the library never retains them after the
 *    call returns.  Host pointers are read or written before the call returns.
 *  - Errors: every call returns a wam_status; no C++ exception crosses this
 *    boundary.  On error the context keeps a message (wam_last_error) and
 *    stays usable unless the status is WAM_ERR_CUDA from a sticky CUDA error.
 */
#ifndef WAM_H
#define WAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WAM_MAX_LEVELS 8

typedef enum {
    WAM_OK = 0,
    WAM_ERR_ARG = -1,      /* invalid argument; nothing was launched */
    WAM_ERR_OOM = -2,      /* device allocation failed */
    WAM_ERR_CUDA = -3,     /* a CUDA call failed */
    WAM_ERR_TIMEOUT = -4,  /* a bounded device wait gave up (a shared-memory image copy of the
                              forward projector did not complete in time); results are invalid */
    WAM_ERR_STATE = -5,    /* call order violated (e.g. no data set) */
    WAM_ERR_IO = -6,       /* a checkpoint file could not be written, read or verified */
    WAM_WARN_NONMONOTONE = 1 /* reconstruction finished, but the cost rose
                                by more than the rounding band at least once */
} wam_status;

enum { WAM_PARALLEL2D = 0, WAM_FAN2D_FLAT = 1, WAM_CONE3D_FLAT_CIRCULAR = 2 };

/* Scan geometry (Sec. II names H only abstractly; the scan is ours). */
typedef struct {
    int kind;                 /* WAM_PARALLEL2D, WAM_FAN2D_FLAT or WAM_CONE3D_FLAT_CIRCULAR */
    int nx, ny, nz;           /* voxels; nz = 1 for 2-D */
    double vx, vy, vz;        /* voxel size, mm */
    int n_views;
    double angle0, angle_span;/* rad */
    int n_bins, n_rows;       /* n_rows = 1 for 2-D */
    double bin_pitch, row_pitch; /* mm on the detector */
    double sod, sdd;          /* fan beam: source-origin, source-detector, mm */
} wam_geometry;

/* Reconstruction schedule (Algorithm 1 + the Results section's tree growth). */
typedef struct {
    int levels;               /* Haar levels L, 0..WAM_MAX_LEVELS (ignored if full_am) */
    int dims;                 /* 2 (2-D Haar; per z-slice for cone beam) or 3 (3-D Haar) */
    int n_iters;              /* J */
    int n_expand;             /* number of tree expansions */
    const int* expand_at;     /* host [n_expand]: expand after this many iterations */
    const double* tau;        /* host [n_expand]: threshold factor; < 0 = every leaf */
    int zsum_criterion;       /* cone beam, dims 2: 1 = expansion criterion summed over z */
    int precision;            /* 32 (FP32 bulk) or 64 (FP64 everywhere) */
    int full_am;              /* 1: plain AM, Omega = I, every pixel active */
    double dmax_clamp;        /* clamp on |Z0 * delta|; <= 0 means 30 */
    int n_subsets;            /* ordered subsets of views (the Conclusion's combination with
                                 ordered subsets): 0 or 1 = none; S > 1: subset s holds the views
                                 k with k mod S = s, and each iteration runs S sub-iterations in
                                 order, each one step of Algorithm 1 on its subset's rays with
                                 that subset's b = Phi_s^T d_s, bhat+- and Z0 (max over its rays).
                                 2-D contexts, wam_reconstruct only; idiv_hist still holds the
                                 full I-divergence at the start of every iteration. */
    int nonneg;               /* plain AM only (full_am, or levels = 0): 1 = keep mu >= 0 by ending
                                 each pixel's (voxel's) step at 0.  With Omega = I the surrogate of
                                 Eq. 1.8 is a sum of one-dimensional convex functions, so this is its
                                 exact minimiser over mu >= 0 and the cost still decreases at every
                                 iteration.  0 (default) = Algorithm 1 as stated, unconstrained.
                                 WAM_ERR_ARG with a Haar tree (levels > 0 and not full_am). */
    double lambda;            /* >= 0.  0 (default): Algorithm 1 as stated (Eq. 1.1 unregularised).
                                 > 0: the regularised problem of Eq. 1.1 with
                                 lambda R(mu) = lambda * sum over the detail coefficients of |beta|
                                 (the wavelet-domain l1 roughness penalty the paper's Summary names).
                                 With the separable surrogate of Eq. 1.8 each detail coefficient's
                                 problem stays one-dimensional and convex: its step is the root of
                                 Eq. 1.9 with b + lambda or b - lambda, whichever lies on its own side
                                 of beta = 0, else beta = 0 exactly; approximations are unpenalised.
                                 idiv_hist then holds I(d || qhat) + lambda * sum |beta_detail|, which
                                 decreases at every iteration.  2-D contexts with levels > 0 and no
                                 ordered subsets (else WAM_ERR_ARG). */
} wam_schedule;

typedef struct wam_ctx wam_ctx;

/* ---- life cycle --------------------------------------------------------- */

/* Create a context for one geometry on the current CUDA device.  The context
 * owns its device buffers (allocated here and on first use by a schedule).
 * Errors: WAM_ERR_ARG for a bad geometry (non-positive sizes; fan beam with
 * the source or the detector line within the image's circumradius of the
 * origin, i.e. SOD <= r or SDD - SOD <= r), WAM_ERR_OOM, WAM_ERR_CUDA. */
wam_status wam_create(const wam_geometry* g, wam_ctx** out);

/* Free every device buffer and the context.  NULL is ignored. */
void wam_destroy(wam_ctx* ctx);

/* Message of the last error on this context ("" if none).  Owned by ctx. */
const char* wam_last_error(const wam_ctx* ctx);

/* Bytes of a tree mask for L levels (sum over l = 1..L of (ny>>l)(nx>>l)). */
size_t wam_mask_bytes(const wam_ctx* ctx, int levels);

/* The same for a schedule's dims: 3 gives the 3-D Haar tree of a cone-beam
 * context (sum of (nz>>l)(ny>>l)(nx>>l)); otherwise wam_mask_bytes. */
size_t wam_mask_bytes_dims(const wam_ctx* ctx, int levels, int dims);

/* ---- data --------------------------------------------------------------- */

/* Set the counts d [n_views][n_bins] (>= 0, finite) and the incident counts
 * I0 (> 0): one value if I0_is_scalar, else one per ray.  With on_device = 0
 * both are host arrays, copied in; with on_device = 1 they are device
 * arrays.  Precomputes d log(d / I0) - d per ray (the cost's constant part,
 * Sec. II footnote).  Errors: WAM_ERR_ARG for negative or non-finite d,
 * I0 <= 0. */
wam_status wam_set_data(wam_ctx* ctx, const float* d, const float* I0, int I0_is_scalar,
                        int on_device, void* stream);

/* ---- the whole method ---------------------------------------------------- */

/* Algorithm 1 (or plain AM when sched->full_am): starting from beta = 0,
 * run sched->n_iters iterations, expanding the tree after the listed
 * iterations.  Outputs (any may be NULL):
 *   mu_out    [nx*ny] final image mu = Omega beta; float* when precision 32,
 *             double* when 64; host or device per on_device
 *   idiv_hist [n_iters + 1] I(d || qhat^(j)), j = 0..n_iters, FP64, host or
 *             device per on_device (entry j is the cost before update j; the
 *             last one is the cost of the final image)
 *   mask_out  [wam_mask_bytes_dims(L, dims)] final tree, host or device per
 *             on_device
 * Returns WAM_WARN_NONMONOTONE when some cost exceeded its predecessor by
 * more than 1e-6 relative (FP32) or 1e-11 (FP64).  Errors: WAM_ERR_STATE if
 * no data were set; WAM_ERR_ARG for a bad schedule (nx, ny not divisible by
 * 2^L, expand_at not increasing, precision not 32/64). */
wam_status wam_reconstruct(wam_ctx* ctx, const wam_schedule* sched, void* mu_out,
                           double* idiv_hist, unsigned char* mask_out, int on_device,
                           void* stream);

/* Many independent scans (bags) of any sizes with one schedule, 2-D contexts,
 * precision 32.  Their iterations are interleaved: all bags share the
 * schedule, so between two expansions every bag runs on the same tree epoch.
 *   use_graph = 0: every bag's kernels are launched directly, bag after bag;
 *   use_graph = 1: one iteration of every bag (each bag on its own stream,
 *     forked from and joined into `stream`) is captured once per epoch into a
 *     CUDA graph that is then launched once per iteration of the epoch (a
 *     device-side counter places each iteration's cost);
 *   use_graph = 2: one iteration of all bags is five kernels, captured once per
 *     epoch: the cell images of every bag, the forward projection of every bag
 *     and the back-projection of every bag by persistent CTAs (about one wave)
 *     that take work items (bag, view, bin tile) and (bag, CTA of the bag's
 *     plan) from a global counter, the bags in decreasing order of work, then
 *     every bag's cost sum and update.  Epochs in which some bag walks its
 *     tree leaf by leaf, or lambda > 0, run as use_graph = 1.
 * Modes 0 and 1 run every bag's forward with the global-memory walk,
 * whatever staged tile height the context is tuned to (WAM_TUNE_FWD_STAGE_ROWS
 * is chosen for a bag running alone; with the bags' kernels running at the
 * same time the staged tiles' shared memory makes them slower), which changes
 * no result: the two walks agree bit for bit.
 * Results of modes 0 and 1 equal n calls of wam_reconstruct bit for bit;
 * mode 2 runs the same kernel bodies and sums in the same order inside other
 * kernels, where the compiler may contract multiply-adds differently: it
 * agrees with them to FP32 rounding.
 *   ctxs      [n] distinct contexts with data set (at most 128 for mode 2)
 *   mu_out    [n] pointers to each bag's image (float, host or device per
 *             on_device), or NULL; hist likewise [n] pointers to n_iters + 1
 *             doubles, or NULL.
 * Returns WAM_WARN_NONMONOTONE if any bag's cost rose; errors as
 * wam_reconstruct (the first failing context keeps the message), WAM_ERR_ARG
 * for use_graph outside 0..2. */
wam_status wam_reconstruct_batch(wam_ctx* const* ctxs, int n, const wam_schedule* sched,
                                 void* const* mu_out, double* const* hist, int on_device,
                                 int use_graph, void* stream);

/* ---- checkpoint / resume ------------------------------------------------- */

/* Algorithm 1 is a fixed-point iteration whose whole state after iteration j
 * is the coefficient vector beta^(j), the tree of active coefficients and the
 * expansions applied so far (b = Phi^T d and Z0 follow from the data and the
 * tree).  wam_checkpoint writes that state for the context's last finished
 * wam_reconstruct (2-D or cone beam): beta (FP64), the tree masks, the cost
 * history I(d || qhat^(0..j)), the schedule it ran, the geometry, CRC-32
 * fingerprints of d and I0, and the back-projector tuning value; the file ends
 * with a CRC-32 of its contents and is written to "<path>.tmp" and renamed.
 * Format (little endian): "WAMCKPT1", u32 version 3, u32 0; 22 int64 (kind,
 * nx, ny, nz, n_views, n_bins, n_rows, levels, dims, zsum_criterion,
 * precision, full_am, n_expand, iterations done, expansions done, N,
 * mask bytes, history length, crc(d), crc(I0), n_subsets, nonneg); 12 double (vx, vy, vz,
 * angle0, angle_span, bin_pitch, row_pitch, sod, sdd, dmax_clamp, tuning, lambda);
 * int64 expand_at[n_expand]; double tau[n_expand]; double beta[N];
 * u8 masks[mask bytes]; double history[iterations done + 1]; u32 crc.
 * Errors: WAM_ERR_STATE if no reconstruction has finished on ctx since its
 * data were set; WAM_ERR_IO if the file cannot be written. */
wam_status wam_checkpoint(wam_ctx* ctx, const char* path);

/* Load a checkpoint into ctx; the next wam_reconstruct on ctx continues from
 * it: it runs iterations j..n_iters - 1 (j = iterations done) and applies the
 * schedule's remaining expansions, and its outputs (image, the full cost
 * history 0..n_iters, tree) equal those of one uninterrupted run bit for bit.
 * The context's back-projector tuning is set to the checkpoint's.  Requires
 * data set (wam_set_data) equal to the checkpoint's (CRC-32 of d and I0) and
 * an equal geometry; the continuing schedule must have the same levels, dims,
 * zsum_criterion, precision, full_am, dmax_clamp, n_subsets, nonneg and lambda, n_iters >= j, and the
 * same first expansions (those applied so far) with no other expansion at or
 * before j, else that wam_reconstruct returns WAM_ERR_STATE and the loaded
 * state stays pending.  wam_set_data discards a pending state.
 * wam_reconstruct_batch refuses contexts with a pending state (WAM_ERR_STATE).
 * Version 2 files (11 doubles, no lambda) are read as lambda = 0.
 * Errors: WAM_ERR_IO for an unreadable, truncated or corrupt file (bad magic,
 * version or CRC); WAM_ERR_STATE for no data or a geometry or data mismatch. */
wam_status wam_resume(wam_ctx* ctx, const char* path);

/* Tuning knobs (set by the caller or by an autotuner that times them). */
enum {
    WAM_TUNE_BACK_CTAS_PER_SM = 1,  /* back-projector launches aim at this many 256-thread CTAs
                                       per SM (default 32, range 0.25 .. 256) by splitting views */
    WAM_TUNE_FWD_STAGE_ROWS = 3,    /* the forward projector's staged image tile: 16, 24 or 32 strips
                                       of 160 cells per shared-memory stage (copied by the tensor
                                       memory accelerator), or 0 (default) = no staging, every ray
                                       reads global memory.  Results are identical for every value
                                       (the same walk and the same order of sums); which is faster
                                       depends on the geometry (an autotuner picks it). */
    WAM_TUNE_GRAPHS = 2             /* 1 (default): wam_reconstruct captures one iteration per tree
                                       epoch (the iterations between two expansions repeat the same
                                       launches) in a CUDA graph and replays it, when no profiling is
                                       on and the run has no ordered subsets; 0: every kernel is
                                       launched directly.  Results are identical either way. */
};
wam_status wam_set_tuning(wam_ctx* ctx, int key, double value);

/* ---- the steps of one iteration (device pointers) ------------------------ */

/* H: p(y) = sum_x h(y|x) mu(x) by exact ray traversal (Sec. II).
 * mu [nx*ny], p [n_views*n_bins].  _f64 takes double arrays. */
wam_status wam_project(wam_ctx* ctx, const float* mu, float* p, void* stream);
wam_status wam_project_f64(wam_ctx* ctx, const double* mu, double* p, void* stream);

/* H^T: g(x) = sum_y h(y|x) s(y), voxel-driven with the same exact h.
 * s [n_views*n_bins], g [nx*ny].  Deterministic (no atomics). */
wam_status wam_backproject(wam_ctx* ctx, const float* s, float* g, void* stream);
wam_status wam_backproject_f64(wam_ctx* ctx, const double* s, double* g, void* stream);

/* Full orthonormal Haar transform with L levels: analysis (inverse = 0,
 * image -> coefficients, Omega^T) or synthesis (inverse = 1, Omega).
 * in, out [nx*ny] FP64, distinct. */
wam_status wam_haar(wam_ctx* ctx, int levels, const double* in, double* out, int inverse,
                    void* stream);

/* a1, Eq. 1.2: mu = Omega beta over the tree: only active coefficients are
 * read (inactive ones are taken as 0).  beta [nx*ny] FP64, masks as above,
 * mu [nx*ny]. */
wam_status wam_synthesize(wam_ctx* ctx, int levels, const unsigned char* masks,
                          const double* beta, float* mu, void* stream);

/* a2+a3, Algorithm 1 first line and Sec. II footnote: for an image mu that is
 * constant on the leaves of the tree (as wam_synthesize produces),
 * qhat(y) = I0(y) exp(-sum_x h(y|x) mu(x)) and the FP64 cost
 * I(d || qhat).  The projection visits one leaf block at a time.  masks = NULL
 * treats every pixel as a leaf.  qhat [n_views*n_bins]; cost: one double in
 * device memory.  Needs wam_set_data. */
wam_status wam_forward(wam_ctx* ctx, int levels, const unsigned char* masks, const float* mu,
                       float* qhat, double* cost, void* stream);
wam_status wam_forward_f64(wam_ctx* ctx, int levels, const unsigned char* masks,
                           const double* mu, double* qhat, double* cost, void* stream);

/* a4, Eq. 1.10: bhat+(z) = sum over rays with phi(y|z) > 0 of qhat(y) phi(y|z)
 * and bhat-(z) over phi < 0, for every active z, phi = H Omega computed per
 * (ray, block) from exact chords through the block's four children.  qhat
 * must be >= 0 (as wam_forward makes it): the two parts come from the sums of
 * qhat phi and qhat |phi|, each clamped to its sign.
 * Inactive entries are set to 0.  bplus, bminus [nx*ny] FP64 in coefficient
 * layout.  levels = 0 gives H^T qhat in bplus (pixel basis). */
wam_status wam_split_backproject(wam_ctx* ctx, int levels, const unsigned char* masks,
                                 const float* qhat, double* bplus, double* bminus, void* stream);

/* a5, Eq. 1.61: Z0 = max_y sum_{z active} |phi(y|z)|; one double written to
 * device memory. */
wam_status wam_z0(wam_ctx* ctx, int levels, const unsigned char* masks, double* z0,
                  void* stream);

/* a6, Eq. 1.9 / Algorithm 1 inner loop: for every active z, beta(z) +=
 * Delta, Delta the zero of b - bhat+ e^{-Z0 Delta} - bhat- e^{Z0 Delta}
 * (stable quadratic root; |Z0 Delta| clamped to `clamp`, <= 0 means 30).
 * b, bplus, bminus, beta [nx*ny] FP64 coefficient layout; z0 a device
 * double.  Inactive entries of beta are untouched. */
wam_status wam_update(wam_ctx* ctx, int levels, const unsigned char* masks, const double* b,
                      const double* bplus, const double* bminus, const double* z0, double clamp,
                      double* beta, void* stream);

/* a6 per coefficient, exactly as wam_reconstruct computes it: Delta(z) =
 * beta~(z) - betahat(z), the zero of Eq. 1.9 (the step of Algorithm 1's inner
 * loop) from b(z), bhat+(z) >= 0 >= bhat-(z), clamped to |Z0 Delta| <= clamp
 * (<= 0 means 30).  precision 32: the FP32 reconstruction's root, i.e.
 * bhat+- rounded to float (they are FP32 sums there), the root in FP32 on
 * inputs divided by max(|b|, bhat+, -bhat-), times an FP32 1/Z0; precision
 * 64: the FP64 root.  lambda > 0: the step of a detail coefficient under the
 * L1 penalty of wam_schedule.lambda, from its current value beta (where the
 * penalised minimiser is beta = 0 exactly, Delta = -beta).  No context is
 * needed.
 *   n         number of coefficients (0 does nothing)
 *   b, bplus, bminus   device [n] FP64
 *   beta      device [n] FP64 current values (read only when lambda > 0; may be NULL otherwise)
 *   lambda    >= 0
 *   z0        Z0 > 0 (Eq. 1.61)
 *   delta     device [n] FP64 output
 *   at_clamp  device [n] int output (1 where the step sits at the clamp), or NULL
 * Errors: WAM_ERR_ARG (null pointer, precision not 32/64, Z0 not positive
 * and finite, lambda negative or not finite), WAM_ERR_CUDA. */
wam_status wam_am_delta(long long n, const double* b, const double* bplus, const double* bminus,
                        const double* beta, double lambda, double z0, double clamp, int precision, double* delta,
                        int* at_clamp, void* stream);

/* a7, Results section: one tree expansion.  Every pixel with S > tau * max S
 * (compared in FP64; tau < 0 selects every pixel) expands its current leaf
 * (read from mask_in) by one level.  S [nx*ny]; mask_in, mask_out distinct
 * device arrays of wam_mask_bytes(levels). */
wam_status wam_expand(wam_ctx* ctx, int levels, const float* S, double tau,
                      const unsigned char* mask_in, unsigned char* mask_out, void* stream);

/* ---- operators of the full Haar basis and gradients ----------------------- */
/* These treat every coefficient of the L-level basis as active (the full
 * tree) and use FP32 device arrays in the coefficient layout above.  They
 * serve differentiation through the method; calls on one context must not
 * overlap (they share the context's work buffers). */

/* p = Phi beta = H Omega beta (Sec. II, Eq. 1.2).  beta [nx*ny], p [V*B]. */
wam_status wam_project_coef(wam_ctx* ctx, int levels, const float* beta, float* p, void* stream);

/* g = Phi^T s = Omega^T H^T s.  s [V*B], g [nx*ny]. */
wam_status wam_backproject_coef(wam_ctx* ctx, int levels, const float* s, float* g, void* stream);

/* Value and gradient of L(beta) = I(d || I0 exp(-Phi beta)) + lambda *
 * sum over detail coefficients of |beta| (the data term of Eq. 1.1 in the
 * wavelet domain of Eq. 1.3, plus an L1 penalty on the details):
 * dL/dbeta = Phi^T (d - qhat) + lambda sign(beta_detail).  loss: one device
 * double (FP64 sum); grad [nx*ny]; qhat [V*B] optional output (may be NULL).
 * Needs wam_set_data.  Errors: WAM_ERR_ARG for lambda < 0 or non-finite. */
wam_status wam_idiv_grad(wam_ctx* ctx, int levels, const float* beta, float lambda, double* loss,
                         float* grad, float* qhat, void* stream);

/* Derivatives of the AM step Delta(b, bhat+, bhat-) of Eq. 1.9 with respect
 * to bhat+ and bhat- (FP64 arithmetic): with u the positive root,
 * dDelta/dbhat+ = u / (Z0 sqrt(b^2 - 4 bhat+ bhat-)),
 * dDelta/dbhat- = 1 / (Z0 u sqrt(b^2 - 4 bhat+ bhat-)); 0 where the step is
 * clamped or degenerate.  b, bplus, bminus [nx*ny] FP64, z0 device double;
 * dplus, dminus [nx*ny] FP32. */
wam_status wam_am_derivs(wam_ctx* ctx, int levels, const double* b, const double* bplus,
                         const double* bminus, const double* z0, double clamp, float* dplus,
                         float* dminus, void* stream);

/* wam_project_coef / wam_backproject_coef over a batch of n vectors in one
 * call: beta [n][nx*ny] -> p [n][n_views*n_bins], s [n][n_views*n_bins] ->
 * g [n][nx*ny], FP32 device, items run one after another on `stream`.
 * WAM_ERR_ARG for n < 0; otherwise the single call's errors. */
wam_status wam_project_coef_batch(wam_ctx* ctx, int levels, int n, const float* beta, float* p, void* stream);
wam_status wam_backproject_coef_batch(wam_ctx* ctx, int levels, int n, const float* s, float* g, void* stream);

/* The loss and gradient of wam_idiv_grad for a batch of n coefficient
 * vectors in one call (the items run one after another on `stream`, on the
 * context's work buffers).  beta, grad [n][nx*ny] FP32; loss [n] FP64 (all
 * device).  Errors as wam_idiv_grad; WAM_ERR_ARG for n < 0. */
wam_status wam_idiv_grad_batch(wam_ctx* ctx, int levels, int n, const float* beta, float lambda, double* loss,
                               float* grad, void* stream);

/* a0, Eq. 1.6 / Algorithm 1's precompute: b(z) = sum_y d(y) phi(y|z) for every
 * coefficient z of the L-level basis, formed as wam_reconstruct forms it in
 * an FP32 run (the pixel back-projection H^T d in FP32 partials summed into
 * FP64, then the FP64 Haar analysis Omega^T).  b [nx*ny] FP64 device, coefficient
 * layout.  Needs wam_set_data. */
wam_status wam_precompute_b(wam_ctx* ctx, int levels, double* b, void* stream);

/* The transposed Jacobian of one AM step on the full tree (Algorithm 1's
 * update of every coefficient, Z0 fixed) applied to gbar: with qhat, bhat+-
 * the quantities of the step at beta (Eq. 1.10) and D+- the derivatives of
 * its root (wam_am_derivs),
 *   gout = gbar - Phi^T [ qhat * (Phi+ (D+ gbar) + Phi- (D- gbar)) ],
 * the chain rule through qhat = I0 exp(-Phi beta) (the step's own identity
 * term is gbar).  beta, b [nx*ny] FP64, z0 device double, gbar, gout
 * [nx*ny] FP32 (distinct), all device; clamp as for wam_update.  Needs
 * wam_set_data. */
wam_status wam_am_step_vjp(wam_ctx* ctx, int levels, const double* beta, const double* b, const double* z0,
                           double clamp, const float* gbar, float* gout, void* stream);

/* out(y) = qhat(y) * sum_z [max(phi(y|z), 0) gbar(z) dplus(z) +
 * min(phi(y|z), 0) gbar(z) dminus(z)] over every z of the full basis: the
 * projection through the positive and negative parts of Phi used by
 * Eq. 1.10, here to apply the transposed Jacobian of bhat+-(beta).
 * qhat may be NULL (factor 1).  gbar, dplus, dminus [nx*ny], out [V*B]. */
wam_status wam_phi_split_project(wam_ctx* ctx, int levels, const float* gbar, const float* dplus,
                                 const float* dminus, const float* qhat, float* out, void* stream);

/* ---- back-projection without device allocation ---------------------------- */

/* Size of the library's fixed device scratch used by wam_backproject_static. */
#define WAM_STATIC_SCRATCH_BYTES (8u << 20)

/* H^T s like wam_backproject, for callers that cannot allocate device memory:
 * a host application that reserves all of its device memory in a fixed pool
 * at start-up and forbids any later cudaMalloc (a serving process with a hard
 * memory budget, or a plug-in whose host owns the device allocator).  The
 * paper has no counterpart to this call; it is a deployment convenience.
 *   g    scan geometry (as for wam_create; 2-D kinds only); no context is needed
 *   s    device [n_views * n_bins] float sinogram, caller-owned
 *   out  device [nx * ny] float image, caller-owned
 * The per-view table and the partial sums live in one static device array of
 * WAM_STATIC_SCRATCH_BYTES (8 MiB) that every GPU which loads the library
 * keeps until the process exits.  The call needs 8 V bytes (rounded up to
 * 256) plus 4 * nx * ny * (number of view ranges) bytes of it; a geometry that
 * needs more is rejected with WAM_ERR_ARG (at most about 1.9 Mpixel images).
 * Nothing is allocated or freed: no cudaMalloc, cudaFree or allocating
 * library routine is called, and no host memory is copied to the device (the
 * view table is computed by a kernel).  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls on a
 * device share the array and it keeps the last call's contents (every entry a
 * call reads is written by that call first): calls that overlap on the GPU,
 * on different streams or threads, race and must be serialised by the
 * caller.  Errors: WAM_ERR_ARG (a geometry wam_create would reject, a
 * cone-beam geometry, a null pointer, scratch too small), WAM_ERR_CUDA. */
wam_status wam_backproject_static(const wam_geometry* g, const float* s, float* out, void* stream);

/* ---- measurement ---------------------------------------------------------- */

/* Kernel classes timed by wam_profile. */
enum {
    WAM_K_FORWARD = 0,     /* ray-driven projection + Beer's law + cost terms */
    WAM_K_BACKPROJECT = 1, /* voxel-driven (split) back-projection */
    WAM_K_UPDATE = 2,      /* partial-sum reduction + AM update */
    WAM_K_Z0 = 3,          /* Z0 row sums */
    WAM_K_SYNTH = 4,       /* tree-masked synthesis */
    WAM_K_TREE = 5,        /* expansion criterion, leaf map, block lists, Haar */
    WAM_NKERNEL = 6
};

typedef struct {
    double ms[WAM_NKERNEL];                /* summed device time (CUDA events), ms */
    unsigned long long launches[WAM_NKERNEL];
    /* counted work: FORWARD = ray-cell intersections with a nonzero chord
     * (cells of the walked grid, or leaf blocks for the leaf walk),
     * BACKPROJECT = ray-child (or ray-block) chords with nonzero length,
     * UPDATE = coefficient steps that sit at the clamp |Z0 Delta| = dmax_clamp
     * (the degenerate roots of Eq. 1.9); other classes 0 */
    unsigned long long work[WAM_NKERNEL];
} wam_stats;

/* Profiling modes of wam_profile. */
enum {
    WAM_PROFILE_OFF = 0,
    WAM_PROFILE_ALL = 1,   /* events and work counters */
    WAM_PROFILE_TIME = 2,  /* events only: the kernels run as unprofiled */
    WAM_PROFILE_WORK = 3   /* work counters only (they add instructions to the kernels) */
};

/* A mode other than WAM_PROFILE_OFF resets the statistics; from then on every
 * kernel launch of wam_reconstruct (and the projections and back-projections
 * of wam_project_coef, wam_backproject_coef and wam_idiv_grad) is bracketed
 * with CUDA events on its stream (ALL, TIME; two event records per launch)
 * and/or counts its work (ALL, WORK: ray-cell intersections with a nonzero
 * chord); WAM_PROFILE_OFF stops.  Errors: WAM_ERR_ARG for an unknown mode. */
wam_status wam_profile(wam_ctx* ctx, int enable);

/* Statistics gathered since wam_profile(ctx, 1); synchronises the stream
 * of the last profiled call.  out must not be NULL. */
wam_status wam_get_stats(wam_ctx* ctx, wam_stats* out);

/* Number of CUDA kernels this library has launched in this process. */
unsigned long long wam_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* WAM_H */
