/*
 * gs.h -- C ABI of the GB300 (sm_103a) differentiable 3D-Gaussian rasterizer used by
 * the tracking and mapping steps of "Visual SLAM with 3D Gaussian Primitives and Depth
 * Priors Enabling Novel View Synthesis" (arXiv 2408.05635).
 *
 * Conventions shared by every entry point
 *   - Plain C types only.  "device" pointers are CUDA global memory of the current
 *     device; "host" pointers are ordinary CPU memory read during the call.
 *   - The caller owns every buffer (inputs, outputs, workspace).  The library owns only
 *     the opaque context, which holds settings, the bound workspace layout and cached
 *     CUDA graphs.  The library never allocates device memory.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls enqueue work
 *     and return without synchronising, except gs_sync_status.
 *   - Errors are returned as gs_status; gs_last_error(ctx) gives a one-line message.
 *     Nothing is thrown and nothing aborts.  Conditions only the device can see
 *     (capacity overflow, an expired bounded wait) are latched in the workspace from
 *     the start of the last gs_project / gs_track_step (which clear them) and
 *     reported by gs_sync_status.
 *   - Images are planar FP32: colour is 3 x H x W, depth and silhouette H x W, pixel
 *     (u, v) at index v * W + u and sampled at its centre (u, v).  With several views
 *     the per-view planes are concatenated in view order: view k starts at pixel
 *     offset P_k = sum_{j<k} W_j H_j (colour at 3 P_k).
 *   - A pose is 7 doubles [qw, qx, qy, qz, tx, ty, tz]: the world->camera rotation
 *     R_{c,w} (unit quaternion, renormalised on read) and translation t_{c,w}, so a
 *     world point X maps to R X + t (Sec. II-A).  Camera axes: x right, y down, z forward.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1, /* a pointer, size or setting is out of range */
    GS_ERR_CUDA = 2,        /* a CUDA runtime call failed (message in gs_last_error) */
    GS_ERR_OOM = 3,         /* host memory for the context could not be allocated */
    GS_ERR_WORKSPACE = 4,   /* workspace missing, too small or misaligned (256 B) */
    GS_ERR_CAPACITY = 5,    /* device saw more pairs or records than the capacities */
    GS_ERR_TIMEOUT = 6,     /* a bounded device-side wait expired */
    GS_ERR_UNSUPPORTED = 7, /* valid request this build does not implement */
    GS_ERR_STATE = 8        /* call order violated (e.g. gs_forward before gs_project) */
} gs_status;

/* Storage type of the per-Gaussian attributes other than the means. */
typedef enum { GS_F32 = 0, GS_BF16 = 1, GS_F16 = 2 } gs_dtype;

typedef struct gs_ctx gs_ctx;

/* The map: n anisotropic Gaussians (Eq. 1 with the covariance Sigma = R s s^T R^T).
 * All arrays device, row-major, n rows.  means: float32 n x 3 (world frame, metres);
 * quats n x 4 (w, x, y, z), any non-zero norm; log_scales n x 3 (scale = exp);
 * opacity_logits n (opacity o = sigmoid); rgb n x 3.  The last four use dtype_attr.
 * Isotropic Gaussians (Eq. 1 as written, eight values each: centre, radius, opacity,
 * colour): quats NULL and log_scales n x 1 (radius = exp); Sigma = r^2 I.  Their
 * gradients fill log_scales as n x 1 and leave the quats gradient untouched. */
typedef struct {
    const float *means;
    const void *quats;
    const void *log_scales;
    const void *opacity_logits;
    const void *rgb;
    int32_t dtype_attr; /* gs_dtype */
    int32_t reserved;
    int64_t n;
} gs_gaussians;

/* Gradients w.r.t. the raw parameters, FP32 device arrays with the shapes above.
 * Every call ADDS into them (sum over views); zero them first.  Any may be NULL. */
typedef struct {
    float *means;
    float *quats;
    float *log_scales;
    float *opacity_logits;
    float *rgb;
} gs_gaussians_grad;

/* Pinhole intrinsics of pi_m (Sec. II-A) and the image size. */
typedef struct {
    double fx, fy, cx, cy;
    int32_t width, height;
} gs_camera;

/* One RGB-D observation per view (planar FP32, device).  depth 0 = no measurement;
 * depth_prior may be NULL (no prior term) and 0 marks a hole. */
typedef struct {
    const float *rgb;
    const float *depth;
    const float *depth_prior;
} gs_targets;

/* Renderer, loss and pose-optimiser settings.  The paper states none of these values;
 * gs_default_config fills the readings documented beside each field. */
typedef struct {
    int32_t tile_w, tile_h; /* initial screen tile of the context's launch schedule
                               (gs_schedule; 16 x 16)                                  */
    float alpha_min;        /* a Gaussian with alpha < alpha_min is skipped (1/255)    */
    float alpha_max;        /* alpha = min(alpha_max, o G) (0.99)                      */
    float t_min;            /* stop before the Gaussian that takes T below t_min (1e-4)*/
    float dilation;         /* eps added to the diagonal of Sigma' in px^2 (0)         */
    float z_near;           /* Gaussians with camera depth <= z_near are dropped (0.2) */
    float jac_clip;         /* J of Sigma' is taken at the mean's image-plane tangent
                               clamped to +-jac_clip * (W / 2 fx, H / 2 fy); no gradient
                               flows through a clamped coordinate; 0 disables (1.3)   */
    float sil_thresh;       /* loss mask: S > sil_thresh and depth > 0 (0.99)          */
    float w_rgb, w_depth, w_vis, w_prior; /* loss weights (0.5, 1, 0.1, 0.5)           */
    double lr_rot, lr_trans;              /* Adam step sizes, rad and m (2e-3, 2e-3)   */
    double beta1, beta2, eps;             /* Adam moments (0.9, 0.999, 1e-8)           */
} gs_config;

/* Sizes that fix the workspace layout. */
typedef struct {
    int64_t n_gaussians;       /* upper bound on gs_gaussians.n of the calls that use it */
    int32_t n_views;           /* V >= 1 views rendered together                         */
    int32_t reserved;
    const gs_camera *cameras;  /* host array of n_views cameras                          */
    int64_t pair_capacity;     /* max (Gaussian, tile) pairs summed over views (< 2^32)  */
    int64_t record_capacity;   /* reserved, must be 0 (every (Gaussian, view) pair has a
                                  record slot in the workspace)                          */
} gs_problem;

/* Counters read back by gs_sync_status. */
typedef struct {
    int64_t n_records; /* visible (Gaussian, view) pairs of the last projection        */
    int64_t n_pairs;   /* (Gaussian, tile) pairs of the last projection                */
    uint32_t err_flags;/* bit 1 pair overflow, bit 2 timeout (bit 0 unused)            */
    uint32_t reserved;
    int64_t fwd_evals;   /* (pixel, Gaussian) footprints evaluated by the last forward    */
    int64_t fwd_contrib; /* ... of which contributed to Eqs. 2-4                          */
    int64_t bwd_evals;   /* footprints evaluated by the last backward                     */
    int64_t bwd_contrib; /* ... of which were differentiated                              */
    uint32_t max_tile;   /* longest per-tile list of the last projection                  */
    uint32_t reserved2;
} gs_counts;

/* ------------------------------------------------------------------ context */

/* Fill cfg with the default readings listed in gs_config. */
void gs_default_config(gs_config *cfg);

/* Create a context with a copy of cfg (NULL = defaults).  *out receives the handle.
 * Errors: GS_ERR_INVALID_ARG (bad setting or NULL out), GS_ERR_UNSUPPORTED (a tile shape
 * outside the set gs_schedule lists), GS_ERR_OOM, GS_ERR_CUDA. */
gs_status gs_create(gs_ctx **out, const gs_config *cfg);

/* Destroy a context (NULL is allowed).  Waits for nothing: the caller must make sure no
 * work enqueued through it is still running if it also frees the workspace. */
gs_status gs_destroy(gs_ctx *ctx);

/* Message of the last error on this context ("" if none); valid until the next call. */
const char *gs_last_error(const gs_ctx *ctx);

/* Name of a status code. */
const char *gs_status_string(gs_status s);

/* Bytes of device workspace the calls below need for `prob` (about 96 B per
 * (Gaussian, view) pair, 12 B per pair capacity, 28 B per pixel).  Errors: INVALID_ARG
 * (NULL argument, n_views < 1, a camera with a non-positive size or focal length,
 * n_gaussians * n_views too large for 32-bit record indices, pair_capacity outside
 * [1, 2^32), record_capacity not 0). */
gs_status gs_workspace_size(const gs_ctx *ctx, const gs_problem *prob, size_t *bytes);

/* ------------------------------------------------------------------ the hot path */

/* Projection and tile binning (forward half of Sec. II-C / Sec. III-B rendering).
 * For every view k and Gaussian i: camera-frame mean R_k x_i + t_k; drop it when its
 * depth is <= z_near; Sigma = Rg diag(s^2) Rg^T; Sigma' = J W Sigma W^T J^T (+ dilation);
 * mu' = pi_m; o = sigmoid(logit); the opacity-aware support o exp(-d^2/2) >= alpha_min;
 * then one (tile, depth) entry for every tile the support ellipse meets (tiles of the
 * context's schedule, 16 x 16 by default).
 * poses: device, n_views x 7 doubles, read on the device when the kernels run.
 * ws: device workspace of at least gs_workspace_size bytes, 256-byte aligned; it
 * holds the projected state that gs_forward / gs_backward consume.  The Gaussian
 * arrays, poses and workspace must stay valid and unchanged until the matching
 * gs_backward has run.  Errors: INVALID_ARG, WORKSPACE, CUDA. */
gs_status gs_project(gs_ctx *ctx, const gs_problem *prob, const gs_gaussians *g, const double *poses, void *ws,
                     size_t ws_bytes, void *stream);

/* Depth sort per tile and front-to-back compositing of colour (Eq. 2), depth (Eq. 3,
 * d_i = camera-frame depth of the mean) and silhouette (Eq. 4) of the views projected
 * by the last gs_project.  rgb / depth / sil: device outputs (planar, concatenated
 * views), each may be NULL.  With targets != NULL the combined loss of Sec. III-B
 *   L = w_rgb sum_M |C - C*|_1 + w_depth sum_M |D - D*| + w_vis sum_{D*>0} (1 - S)
 *     + w_prior sum_{M, prior>0} |D - prior|,   M = {S > sil_thresh, D* > 0}
 * is evaluated in the same kernel: loss (device, n_views doubles, may be NULL)
 * receives it per view and its gradient w.r.t. the rendered maps is kept in the
 * workspace for gs_backward.  Errors: STATE (no projection bound), CUDA. */
gs_status gs_forward(gs_ctx *ctx, const gs_targets *targets, float *rgb, float *depth, float *sil, double *loss,
                     void *stream);

/* Reverse compositing and chain rule (the differentiable rendering of Sec. III-B and
 * Sec. III-C).  Upstream gradients: either all three of d_rgb / d_depth / d_sil
 * (device, planar like gs_forward's outputs) or all three NULL to use the gradient of
 * the loss evaluated by the last gs_forward.  grads (NULL = none) receive, ADDED, the
 * gradients w.r.t. every Gaussian parameter summed over views.  pose_grad (device,
 * n_views x 6 doubles, may be NULL) is OVERWRITTEN with (d theta, d t) per view, reduced
 * in FP64: theta turns the camera about its own centre (camera-frame points
 * x_c <- Exp(theta) x_c) and t shifts them (x_c <- x_c + t).
 * One gs_backward per gs_project (the projection clears the per-Gaussian accumulators).
 * Errors: INVALID_ARG (partly NULL upstream), STATE (no projection, or its gradients
 * were already taken), CUDA. */
gs_status gs_backward(gs_ctx *ctx, const float *d_rgb, const float *d_depth, const float *d_sil,
                      gs_gaussians_grad *grads, double *pose_grad, void *stream);

/* `iters` tracking iterations (Sec. III-B): each renders every view at its current
 * pose, evaluates the combined loss against `targets`, back-propagates to the pose
 * only and applies the decoupled rotation / translation Adam step in FP64 on the
 * device: separate moments for theta and t; the camera turns about its own centre,
 * R <- Exp(-step_theta) R (quaternion renormalised) and t <- Exp(-step_theta) t, then
 * moves, t <- t - step_t.  poses (device, n_views x 7) is updated in place;
 * adam_state (device, n_views x 16 doubles: m_rot 3, v_rot 3, m_t 3, v_t 3, step
 * count, beta1^k, beta2^k, 1 unused; zero it to start) carries the moments; loss_hist (device,
 * iters x n_views doubles, may be NULL) receives the loss before each update.  The
 * iterations are replayed from a CUDA graph that the context builds once per
 * argument set; no host synchronisation, no allocation.
 * Errors: INVALID_ARG (iters < 1 or NULL), WORKSPACE, CUDA. */
gs_status gs_track_step(gs_ctx *ctx, const gs_problem *prob, const gs_gaussians *g, const gs_targets *targets,
                        double *poses, double *adam_state, double *loss_hist, int32_t iters, void *ws,
                        size_t ws_bytes, void *stream);

/* The host side of gs_track_step_upload, all page-locked host memory (cudaHostAlloc,
 * cudaHostRegister): the frame's targets laid out like gs_targets (rgb 3 x P, depth P,
 * depth_prior P or NULL), and result (NULL, or n_views x 8 doubles mapped into the
 * device's address space) receiving each view's pose after the last iteration (7) and its
 * loss before the last update (1), stored by the device at the end of the call. */
typedef struct {
    const float *rgb;
    const float *depth;
    const float *depth_prior;
    double *result;
} gs_host_targets;

/* gs_track_step for a frame that is still in host memory.  With `targets` (device
 * buffers, which it overwrites) the call first copies src into them, on a branch of its
 * work that runs beside the first iteration's projection, scan and key emission; the
 * first compositor waits for the copy, everything else is gs_track_step.  With targets
 * NULL there is no copy: the kernels read the frame in place through the device
 * addresses of src's arrays (page-locked memory mapped into the device's address space,
 * read over the host link by the compositor: each block loads its pixels' targets once
 * its first batch is staged, so the reads overlap its forward walk) -- the faster form for
 * one iteration, while a copy is read from device memory by every iteration of a longer
 * call.  The copy or the
 * in-place reads are part of the CUDA graph (one per argument set, src included).  With
 * src->result the poses and losses reach host memory without a copy after the call (the
 * finalize kernel stores them there); they are valid once the stream has passed the call.
 * Errors: as gs_track_step; INVALID_ARG when src is NULL, lacks rgb or depth, has a depth
 * prior exactly when targets has none (or the reverse), or an array is not page-locked
 * host memory (mapped into the device's address space where it is read in place or is
 * the result). */
gs_status gs_track_step_upload(gs_ctx *ctx, const gs_problem *prob, const gs_gaussians *g, const gs_targets *targets,
                               const gs_host_targets *src, double *poses, double *adam_state, double *loss_hist,
                               int32_t iters, void *ws, size_t ws_bytes, void *stream);

/* Synchronise `stream`, read the device counters of the bound workspace into counts
 * (may be NULL) and clear the latched flags.  Returns CAPACITY or TIMEOUT when the
 * device latched one since the last call (results of that call are invalid), STATE
 * when no workspace is bound, CUDA on a runtime error. */
gs_status gs_sync_status(gs_ctx *ctx, void *stream, gs_counts *counts);

/* ------------------------------------------------------------------ instrumentation */

/* Per-kernel device time of the last enqueued work, for profiling. */
typedef struct {
    char name[24]; /* kernel (k_project, k_scan_tiles, k_emit, k_forward, k_backward,
                      k_bproject, k_finalize) */
    float ms;      /* CUDA-event time from the marker before this kernel's launch (which is the
                      end marker of the previous kernel when that one is also marked) to the
                      marker after it */
} gs_kernel_time;

/* Enable (1) or disable (0) CUDA-event markers between the library's kernels on the
 * stream they are launched on (also inside the tracking graph, as event nodes).  Off by
 * default; events are created once per context.  Errors: CUDA. */
gs_status gs_set_profiling(gs_ctx *ctx, int32_t enable);

/* Select the kernels bracketed by profiling markers: bit k of mask selects, in order,
 * k_project, k_scan_tiles, k_emit, k_forward, k_backward, k_bproject, k_finalize (0x7F:
 * all, as gs_set_profiling(ctx, 1); 0: off).  Unselected kernels get no events, so timing
 * one kernel disturbs the launch chain of the others less.  Errors: INVALID_ARG (a bit
 * above 6). */
gs_status gs_set_profiling_mask(gs_ctx *ctx, uint32_t mask);

/* Synchronise on the last marker and return the per-kernel times of the work enqueued
 * by the last gs_project / gs_forward / gs_backward sequence or gs_track_step call (all
 * iterations).  out (host, cap entries) receives min(cap, available) entries; *count the
 * number available.  Errors: STATE (profiling off or nothing recorded), CUDA. */
gs_status gs_kernel_times(gs_ctx *ctx, gs_kernel_time *out, int32_t cap, int32_t *count);

/* Instrumentation of the pose reduction (the FP64 summation the pose gradient of the
 * decoupled update of Sec. III-B asks for): the per-cell partial sums the last pose
 * backward left in the workspace, copied to `out` (host, cap floats) after synchronising
 * `stream`.  Cell c of view v holds six double-float values (hi, lo pairs of FP32), at
 * out[12 (v nblk + c) ..], nblk = ceil(n / 256); the pose gradient is their sum over the
 * view's cells.  *count gets the number of floats (12 V nblk); nothing is copied when
 * cap is smaller.  Errors: INVALID_ARG, STATE (nothing projected), CUDA. */
gs_status gs_pose_partials(gs_ctx *ctx, float *out, int64_t cap, int64_t *count, void *stream);

/* ------------------------------------------------------------------ launch schedule */

/* How the context launches the binning and the two compositors.  Every pixel composites
 * the same Gaussians in the same (depth, index) order under every schedule (a tile's list
 * holds every Gaussian whose support reaches one of its pixels).  The sub-buckets only
 * split where a tile's pairs are counted and placed (the tile's list is sorted whole) and
 * the batch depth only sets how many of a tile's depth-sorted Gaussians the tile block
 * stages into shared memory at a time: with the tile shape fixed, images are bit-identical
 * and gradients differ by FP32 summation order.  The footprints are evaluated relative to
 * the tile origin, so another tile shape changes their rounding (and may flip an
 * alpha_min or t_min decision that sits within rounding of its threshold).  A tile block
 * has one thread per pixel, so the tile shape also sets the threads per tile. */
typedef struct {
    int32_t tile_w, tile_h; /* screen tile in pixels: tile_w in {8, 16, 32}, tile_h in
                               {4, 8, 16, 32}, 64 <= tile_w tile_h <= 256 (16 x 16)    */
    int32_t sub_buckets;    /* counters per tile for the pair count and key emission:
                               1, 2 or 4 (4; fewer are used when tiles x 4 exceeds 2^22) */
    int32_t fwd_batch;      /* Gaussians staged per forward batch: 64, 128 or 256, at
                               most tile_w tile_h (256)                                 */
    int32_t bwd_batch;      /* Gaussians staged per backward batch: the same (256)      */
    int32_t flags;          /* GS_SCHED_* bits (0)                                      */
} gs_schedule;

/* gs_schedule.flags: GS_SCHED_FUSED -- in gs_track_step, each tile's forward with the
 * fused loss and its pose-only reverse walk run in one kernel (k_track_tile): the same
 * arithmetic as the two compositing kernels, with the pixel state kept in registers
 * between the walks and the last forward batch reused by the reverse walk.  Needs
 * fwd_batch == bwd_batch.  Other calls are unaffected. */
#define GS_SCHED_FUSED 1
/* gs_schedule.flags: GS_SCHED_RADIX -- the front-to-back order of Eqs. 2-4 comes from one
 * device-wide LSD radix sort of all (tile, depth) keys (eight-bit digits, stable passes,
 * runs of equal keys then put in Gaussian order) run after the key emission, instead of
 * the per-tile sort inside the forward.  Same order, same results. */
#define GS_SCHED_RADIX 2

/* Read the context's schedule (defaults after gs_create).  Errors: INVALID_ARG (NULL). */
gs_status gs_get_schedule(const gs_ctx *ctx, gs_schedule *out);

/* Set the schedule used by every later call on the context (a cached tracking graph is
 * rebuilt on its next use).  The workspace size does not depend on it (it has room for
 * the tiles of the smallest shape), but a smaller tile can make more (Gaussian, tile)
 * pairs than the problem's pair_capacity holds (reported as CAPACITY by gs_sync_status).
 * Errors: INVALID_ARG (NULL, or a value outside the sets above). */
gs_status gs_set_schedule(gs_ctx *ctx, const gs_schedule *sched);

/* One measurement of gs_autotune. */
typedef struct {
    int32_t stage;        /* 0: tile shape, timed as a whole pass (projection, scan,
                             emission, forward with the fused loss, backward);
                             1: binning (projection, scan, emission) per sub_buckets;
                             2: forward compositing per fwd_batch;
                             3: backward compositing per bwd_batch;
                             4: (pose_only) both compositors, as two kernels or fused
                                (GS_SCHED_FUSED);
                             5: the sort, per tile or device-wide (GS_SCHED_RADIX),
                                timed as a whole pass                                    */
    float ms;             /* mean device time of one pass of the stage (CUDA events on
                             the stream, warm caches, after one untimed pass); -1 when
                             the setting made more pairs than pair_capacity (not timed) */
    gs_schedule schedule; /* the schedule of the timed passes                          */
} gs_tune_entry;

/* Autotuner of the launch schedule for one problem.  On the given Gaussians, poses and
 * targets it times, stage after stage:
 *   - the tile shapes 16 x 16, 32 x 8, 16 x 8 and 8 x 8, one whole pass each (batch
 *     depths capped at the tile's threads);
 *   - every sub-bucket count (the binning);
 *   - every forward batch depth, then every backward batch depth the chosen tile allows
 *     (the pose-only walk of tracking when pose_only != 0, the walk for all Gaussian
 *     parameters otherwise);
 *   - with pose_only, the two compositors as two kernels against the fused tracking
 *     kernel (GS_SCHED_FUSED, both batch depths set to the forward's);
 *   - the per-tile sort against the device-wide radix sort (GS_SCHED_RADIX), one whole
 *     pass each;
 * `reps` passes each.  Each stage starts from the previous stage's choice (first, the
 * context's current schedule) and keeps it unless another setting is at least 1 % faster;
 * the final choice is set on the context.  It uses the workspace (sized by
 * gs_workspace_size for `prob`) as gs_project does and synchronises `stream`, so it
 * cannot be captured into a graph; afterwards no projection is bound (call gs_project or
 * gs_track_step next).  table (host, cap entries, may be NULL) receives the measurements
 * in order, *count (may be NULL) their number (17 at most); best (may be NULL) the chosen
 * schedule.  A setting whose pairs overflow pair_capacity is recorded with ms = -1 and
 * not chosen; an overflow of the context's current schedule is reported as CAPACITY (the
 * schedule is then left unchanged).
 * Errors: INVALID_ARG (as gs_project; targets without rgb or depth; reps outside
 * [1, 1000]; a capturing stream), WORKSPACE, CAPACITY, CUDA. */
gs_status gs_autotune(gs_ctx *ctx, const gs_problem *prob, const gs_gaussians *g, const double *poses,
                      const gs_targets *targets, int32_t pose_only, int32_t reps, void *ws, size_t ws_bytes,
                      gs_tune_entry *table, int32_t cap, int32_t *count, gs_schedule *best, void *stream);

/* ------------------------------------------------------------------ scene optimisation */

/* The map as the scene optimisation holds it (Sec. III-C).  Device arrays with room for
 * `capacity` Gaussians, of which the first n are live; n is a device int64 that the calls
 * below read and update, so a sequence of them needs no host synchronisation.
 *   means, quats, log_scales, opacity_logits, rgb: FP32, the shapes of gs_gaussians, the
 *     optimiser's master copy (a render reads them as a gs_gaussians with GS_F32);
 *   lowp_*: NULL, or a copy of the four attribute arrays in lowp_dtype (GS_BF16 or
 *     GS_F16, rounded to nearest) that every call below refreshes where it changes the
 *     FP32 values, for renders with that dtype (they share the FP32 means);
 *   adam_state: NULL, or the Adam moments, 28 x capacity FP32: the first moments of the
 *     groups means (3 capacity floats), quats (4), log_scales (3), opacity_logits (1),
 *     rgb (3), then the second moments in the same layout; a Gaussian's entries are the
 *     rows of its index in each group.
 * An isotropic map (Eq. 1 as written) has quats = lowp_quats = NULL and log_scales of
 * capacity x 1; its moments are 16 x capacity floats (means 3, log_scales 1,
 * opacity_logits 1, rgb 3, then the second moments).
 * Every pointer must be 16-byte aligned and capacity a multiple of 4. */
typedef struct {
    float *means;
    float *quats;
    float *log_scales;
    float *opacity_logits;
    float *rgb;
    void *lowp_quats;
    void *lowp_log_scales;
    void *lowp_opacity_logits;
    void *lowp_rgb;
    int32_t lowp_dtype; /* gs_dtype of the lowp arrays (ignored when they are NULL) */
    int32_t reserved;
    int64_t capacity;
    float *adam_state;
} gs_map;

/* Settings of the scene optimisation.  The paper gives none; gs_default_map_config fills
 * the readings beside each field. */
typedef struct {
    double lr_means, lr_quats, lr_log_scales, lr_opacity_logits, lr_rgb; /* Adam step sizes per
                                  group (1e-4, 1e-3, 1e-3, 5e-2, 2.5e-3)                    */
    double beta1, beta2, eps;  /* Adam moments and denominator guard (0.9, 0.999, 1e-15)    */
    float sil_add;             /* a keyframe pixel gets a Gaussian where S < sil_add (0.5)  */
    float opacity_min;         /* gs_map_prune drops Gaussians with opacity < this (0.005)  */
} gs_map_config;

void gs_default_map_config(gs_map_config *cfg);

/* Device scratch, in bytes, that gs_map_add (items = the view's pixels) and gs_map_prune
 * (items = the source map's capacity) need. */
size_t gs_map_scratch_bytes(int64_t items);

/* New Gaussians from one RGB-D observation: every Gaussian of the first frame (Sec. III-A)
 * and, on a keyframe, the pixels its silhouette shows as new observations (Sec. III-C; the
 * silhouette is the mask of where Gaussians are added, Sec. V).  A pixel with depth d > 0
 * (and S < sil_add when sil is given) becomes a Gaussian centred on its sample point
 * (u, v) unprojected with d through the pose, with its colour, opacity 0.5 (logit 0), the
 * identity rotation and the isotropic scale d / f, f = (fx + fy) / 2 (one pixel wide in
 * the image).  They are appended after the live Gaussians in row-major pixel order; their
 * Adam moments are zeroed.
 *   cam: host; pose: device, 7 doubles (world->camera); rgb, depth: device planes of the
 *   view; sil: device plane or NULL (every pixel with depth); n: device int64, the live
 *   count, updated; scratch: device, gs_map_scratch_bytes(W H) bytes, 256-byte aligned;
 *   err_flags: device uint32 or NULL, bit 0 set when the map was full (the Gaussians
 *   that fit were added, n = capacity).
 * Errors: INVALID_ARG (NULL or misaligned pointer, bad camera, scratch too small), CUDA. */
gs_status gs_map_add(const gs_map_config *cfg, const gs_map *map, int64_t *n, const gs_camera *cam,
                     const double *pose, const float *rgb, const float *depth, const float *sil, void *scratch,
                     size_t scratch_bytes, uint32_t *err_flags, void *stream);

/* One Adam step on every parameter of the live Gaussians, keyframe poses fixed
 * (Sec. III-C): per group, m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), in FP32.
 *   grads: the gradients of the loss summed over the window (gs_backward's), FP32 device
 *   arrays of capacity rows (rows >= n are not read); map->adam_state is required;
 *   n: device int64 live count; step: t >= 1.
 * Errors: INVALID_ARG, CUDA. */
gs_status gs_map_adam_step(const gs_map_config *cfg, const gs_map *map, const int64_t *n,
                           const gs_gaussians_grad *grads, int64_t step, void *stream);

/* Duplicate removal (Sec. III-C): the live Gaussians of src whose opacity is at least
 * opacity_min (decided on the FP32 logit against logit(opacity_min) rounded to FP32) are
 * copied, in order, to dst with their Adam moments and lowp copies (each moved only where
 * both maps have them); n_dst receives their count.  src and dst must not overlap and
 * dst->capacity must be at least src->capacity.
 *   n_src, n_dst: device int64; scratch: device, gs_map_scratch_bytes(src->capacity).
 * Errors: INVALID_ARG, CUDA. */
gs_status gs_map_prune(const gs_map_config *cfg, const gs_map *src, const int64_t *n_src, const gs_map *dst,
                       int64_t *n_dst, void *scratch, size_t scratch_bytes, void *stream);

/* Image-quality sums of one rendered view against its observation, behind the evaluation
 * of Sec. IV (PSNR of the colour, the average depth error).  rgb / depth: the render,
 * rgb_t / depth_t: the observation, planar FP32 device arrays of `pixels` pixels; out:
 * device, 4 doubles = (sum of squared colour errors over every pixel and channel,
 * sum |D - D*| over the pixels with D* > 0, their count, sum (D - D*)^2 over them),
 * accumulated in FP64 in a fixed order.  Errors: INVALID_ARG, CUDA. */
gs_status gs_image_metrics(const float *rgb, const float *depth, const float *rgb_t, const float *depth_t,
                           int64_t pixels, double *out, void *stream);

/* Device scratch, in bytes, that gs_msssim needs for a width x height image. */
size_t gs_msssim_scratch_bytes(int32_t width, int32_t height);

/* Multi-scale structural similarity (Wang, Simoncelli and Bovik, 2003) of a rendered
 * colour image against its observation, the MS-SSIM of Sec. IV: per scale the mean
 * contrast-structure term (and on the coarsest the mean luminance term) under an 11 x 11
 * Gaussian window (sigma 1.5) at every position where it fits, constants K1 = 0.01,
 * K2 = 0.03 for colours in [0, 1], five scales made by 2 x 2 average pooling (odd last
 * row / column dropped), negative terms clamped at 0, combined with the published
 * exponents (0.0448, 0.2856, 0.3001, 0.2363, 0.1333) per colour channel.
 *   rgb, rgb_t: device, planar 3 x height x width FP32; width and height at least 176 (the
 *   coarsest scale holds one window); out: device, 4 doubles = (mean over the channels,
 *   red, green, blue); scratch: device, gs_msssim_scratch_bytes, 256-byte aligned.
 * Errors: INVALID_ARG, CUDA. */
gs_status gs_msssim(const float *rgb, const float *rgb_t, int32_t width, int32_t height, double *out, void *scratch,
                    size_t scratch_bytes, void *stream);

/* ------------------------------------------------------------------ no-allocation render */

/* Limits of gs_render_static. */
#define GS_STATIC_MAX_GAUSSIANS 65536
#define GS_STATIC_MAX_PIXELS (640 * 480)
#define GS_STATIC_MAX_PAIRS (1 << 19)

/* Render one view -- projection, tile binning, per-tile depth sort and compositing of
 * colour, depth and silhouette, with the combined loss when targets are given -- the
 * same computation as gs_project + gs_forward, but with no workspace and no allocation.
 * The paper has no counterpart: this is for callers that cannot allocate device memory
 * where they render (a plugin or real-time loop inside a host application that owns
 * the memory pool, or code that must not call cudaMalloc / cudaFree because they
 * synchronise the device).  Its scratch (about 24 MB) is a static device array of the
 * library, which every GPU that loads the library holds until the process exits.
 *   cfg: settings (gs_default_config for the defaults); no context is needed.
 *   g: at most GS_STATIC_MAX_GAUSSIANS Gaussians; cam: at most GS_STATIC_MAX_PIXELS
 *   pixels; pose: device, 7 doubles; targets: NULL or an RGB-D observation (loss then
 *   optional); rgb / depth / sil: device outputs, each may be NULL; loss: device, one
 *   double, may be NULL; err_flags: device, one uint32 receiving the device-detected
 *   flags of gs_counts (bit 1: more than GS_STATIC_MAX_PAIRS pairs, output invalid),
 *   may be NULL.
 * The first call on a device looks up the array's device address (with that device
 * current); make it before any stream capture.  Every call uses the same array and the
 * array keeps the last call's contents: calls that overlap on the GPU (different
 * streams, or several host threads) race and corrupt each other's results.  Nothing is
 * allocated, host or device.  Errors: INVALID_ARG (NULL argument, a size above the
 * limits), UNSUPPORTED (tile shape), CUDA. */
gs_status gs_render_static(const gs_config *cfg, const gs_gaussians *g, const gs_camera *cam, const double *pose,
                           const gs_targets *targets, float *rgb, float *depth, float *sil, double *loss,
                           uint32_t *err_flags, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GS_H */
