/*
 * gsplat.h -- C ABI of the GB300 (sm_103a) differentiable 3D Gaussian
 * splatting hot path of GSFusion (arXiv 2408.12677): the tile-based
 * rasterizer forward and backward pass and the Adam update of the Gaussian
 * parameters (Sec. III-B.3 "Online Optimization"), for one view or a batch
 * of views, and the per-frame steps around it: TSDF fusion (Sec. III-B.1,
 * Eq. 6-9), quadtree seeding with the voxel-weight or rendered-alpha
 * novelty check (Sec. III-B.2, Eq. 10), and host-side failure detection.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All array pointers are DEVICE pointers on the context's device, owned by
 *   the caller, unless a comment says "host".  Float arrays are IEEE float32,
 *   contiguous, row-major.  Images are planar: colour [3, H, W], depth, alpha
 *   [H, W].
 * - Calls are asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *   default stream) except where noted.  Inputs must stay valid and
 *   unmodified until the stream reaches the call.
 * - Every function returns a gs_status; nothing is thrown across the ABI.
 *   gs_last_error(ctx) gives a human-readable message for the last failure on
 *   that context.  Argument checks happen on the host before any GPU work:
 *   a call that returns GS_ERR_INVALID_ARG has enqueued nothing.
 * - A context is bound to one device and is not thread-safe; use one context
 *   per host thread.  It owns the scratch memory of the path (projected
 *   features, sort buffers, per-tile ranges, per-pixel state); grow-on-demand
 *   allocations use cudaMalloc.
 * - Camera model (Eq. 4): a point p_w maps to p_c = R p_w + t (the viewmat is
 *   the world-to-camera transform T_CW = T_WC^{-1}, R row-major) and projects
 *   to (fx x/z + cx, fy y/z + cy); pixel (i, j) has its centre at
 *   (i + 0.5, j + 0.5).  Camera x right, y down, z forward.
 * - Gaussian parameters (Eq. 1-2 and Sec. III-A.2), N Gaussians, SH degree
 *   d in {0, 1, 2, 3}, K = (d + 1)^2 coefficients per colour channel:
 *     means [N, 3], log_scales [N, 3] (S = diag(exp(log_s))),
 *     quats [N, 4] (w, x, y, z; normalised inside), opacity_logits [N]
 *     (opacity = sigmoid), sh [N, K, 3] (real SH basis with the
 *     Condon-Shortley phase, colour = max(0, 0.5 + sum_k Y_k(dir) sh_k),
 *     dir = unit vector from the camera centre to the mean).
 *   The flat layout used by gs_adam_step is these five arrays back to back
 *   in that order: N * (11 + 3K) floats.
 */
#ifndef GSPLAT_H
#define GSPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GSPLAT_ABI_VERSION 1

typedef struct CUstream_st *gs_stream_t; /* identical to cudaStream_t */

typedef enum {
  GS_OK = 0,
  GS_ERR_INVALID_ARG = 1, /* bad pointer, size or configuration; nothing enqueued */
  GS_ERR_CUDA = 2,        /* a CUDA runtime call failed (message in gs_last_error) */
  GS_ERR_CAPACITY = 3,    /* (tile, Gaussian) pairs exceeded the reserved capacity in no-sync mode */
  GS_ERR_NONFINITE = 4,   /* non-finite values detected (gs_count_nonfinite) */
  GS_ERR_BOUNDS = 5,      /* the bounds-checked build met an out-of-bounds index (gs_sync_status) */
  GS_ERR_TIMEOUT = 6,     /* reserved: a bounded device wait gave up */
  GS_ERR_OOM = 7,         /* cudaMalloc of context scratch failed */
  GS_ERR_STATE = 8        /* gs_render_bwd without a matching gs_render_fwd on this context */
} gs_status;

typedef struct {
  float fx, fy, cx, cy;   /* pinhole intrinsics in pixels */
  int32_t width, height;  /* image size in pixels, each in [1, 65535 * tile size] */
} gs_camera;

typedef struct {
  float R[9]; /* world-to-camera rotation, row-major */
  float t[3]; /* world-to-camera translation */
} gs_viewmat;

typedef struct {
  const float *means, *log_scales, *quats, *opacity_logits, *sh; /* device, see layout above */
  int64_t n;          /* number of Gaussians, 0 <= n < 2^31 */
  int32_t sh_degree;  /* 0..3 */
} gs_gaussians;

typedef struct {
  float *means, *log_scales, *quats, *opacity_logits, *sh; /* device; gradients are ACCUMULATED (+=) */
} gs_grads;

typedef struct {
  int32_t tile_w, tile_h; /* 16x16, 8x32 or 32x8 */
  int32_t batch;          /* list entries a warp stages per round (one per lane): 32, the only value */
  float bg[3];            /* background colour added with the final transmittance */
  float near_z;           /* cull Gaussians with camera z <= near_z (0.2) */
  float alpha_max;        /* opacity clamp (0.99) */
  float alpha_min;        /* skip contributions below this alpha (1/255) */
  float t_eps;            /* stop before the Gaussian that would push T below this (1e-4) */
  float dilation;         /* added to the 2D covariance diagonal, px^2 (0.3) */
} gs_raster_cfg;

typedef struct {
  float lr_means, lr_log_scales, lr_quats, lr_opacity, lr_sh_dc, lr_sh_rest;
  float beta1, beta2, eps;
  int32_t zero_grads; /* 1: gs_adam_step writes 0 to every gradient it consumed */
} gs_adam_cfg;

typedef struct {
  int64_t n_pairs;          /* (tile, Gaussian) pairs of the last forward pass (-1 in no-sync mode) */
  int64_t pair_capacity;    /* pairs the context can hold without growing */
  int64_t kernel_launches;  /* kernels this context has launched since creation */
  int64_t n_tiles;          /* tiles of the last forward pass */
  int64_t evals_blended;    /* (pixel, Gaussian) pairs blended, summed over forward passes since the last reset */
  int64_t evals_tiled;      /* (pixel, list entry) visits of the forward raster loop, same period */
} gs_stats;

/* Stages timed by the optional profiler (CUDA events on the launch stream). */
typedef enum {
  GS_STAGE_PROJECT_FWD = 0,
  GS_STAGE_DEPTH_SORT,
  GS_STAGE_DUPLICATE,
  GS_STAGE_PAIR_SORT,
  GS_STAGE_RANGES,
  GS_STAGE_RASTER_FWD,
  GS_STAGE_LOSS,
  GS_STAGE_RASTER_BWD,
  GS_STAGE_PROJECT_BWD,
  GS_STAGE_ADAM,
  GS_NUM_STAGES
} gs_stage;

typedef struct gs_ctx gs_ctx;

/* Create a context on CUDA device `device`.  `pair_capacity` pre-sizes the
 * (tile, Gaussian) pair buffers (0 = grow on demand).  *ctx receives the
 * handle.  Sync mode is on: each forward pass reads the pair count back to
 * the host once and grows the pair buffers as needed. */
gs_status gs_ctx_create(gs_ctx **ctx, int device, int64_t pair_capacity);

/* Free the context and all scratch it owns.  Synchronises its device. */
gs_status gs_ctx_destroy(gs_ctx *ctx);

/* Last error message of this context ("" if none).  Owned by the context. */
const char *gs_last_error(const gs_ctx *ctx);

/* Pre-size scratch for up to n_gaussians items (Gaussians times views in a
 * batched call), n_pixels pixels (summed over the views) and n_pairs pairs
 * (each 0 = leave as is), e.g. before capturing a CUDA graph. */
gs_status gs_ctx_reserve(gs_ctx *ctx, int64_t n_gaussians, int64_t n_pixels, int64_t n_pairs);

/* sync = 1 (default): the forward pass reads the pair count to the host and
 * grows buffers.  sync = 0: no host synchronisation inside the forward pass
 * (stream-capturable); pairs beyond the reserved capacity are dropped and
 * the next gs_render_fwd / gs_sync_status reports GS_ERR_CAPACITY.  While
 * every tile list that the context's sync-mode passes have seen is at most
 * 2048 entries long, sync = 0 passes bin into per-tile buckets written by
 * the projection (no scan or scatter launch; the same lists and images),
 * each bucket twice as long as the longest list seen, rounded up to a
 * power of two from 1024 to 4096; a list that outgrows its bucket is
 * reported by gs_sync_status as GS_ERR_CAPACITY, after which the context
 * bins by counting and scatter (a captured graph has to be recaptured). */
gs_status gs_ctx_set_sync(gs_ctx *ctx, int sync);

/* Set the context's device-side Adam step counter (used by
 * gs_render_bwd_adam with step = 0, which increments it before each use).
 * Synchronises the device. */
gs_status gs_ctx_set_adam_step(gs_ctx *ctx, int64_t step);

/* on = 1 (default): the raster passes visit the tiles longest list first
 * (tiles ordered by the length class of their lists, four classes per octave
 * of the length, computed during binning), so the slowest tiles start early
 * and the grid ends evenly; on = 0
 * visits them in index order.  Results do not depend on the order.  Takes
 * effect at the next forward pass. */
gs_status gs_ctx_set_tile_order(gs_ctx *ctx, int on);

/* on = 1 (default): each raster pass is one persistent launch of as many
 * CTAs as the GPU holds at once, whose warps pull (tile, 8 x 8 pixel block)
 * jobs from a device counter in the visit order above, for all views of a
 * batch.  on = 0: one CTA per tile.  Results do not depend on it. */
gs_status gs_ctx_set_persistent(gs_ctx *ctx, int on);

/* Synchronise the stream, then report GS_ERR_BOUNDS if the bounds-checked
 * build met an out-of-bounds index since the last call (see
 * gs_bounds_checked), else GS_ERR_CAPACITY if a no-sync forward pass
 * overflowed the pair buffers or a tile bucket (see gs_ctx_set_sync);
 * clears the flag it reports. */
gs_status gs_sync_status(gs_ctx *ctx, gs_stream_t stream);

/* Counters of this context (host struct).  The two eval counters live on the
 * device: this call synchronises the device when counting is on. */
gs_status gs_get_stats(gs_ctx *ctx, gs_stats *out);

/* counting = 1 makes every forward pass add its blended and visited
 * (pixel, Gaussian) counts to two device counters (one atomic per CTA);
 * also zeroes them.  Off by default. */
gs_status gs_set_eval_counting(gs_ctx *ctx, int counting);

/* profiling = 1: record a CUDA event pair around every stage launched on the
 * call's stream and accumulate the elapsed times; also clears the totals.
 * gs_profile_read synchronises the device and returns, per gs_stage, the
 * summed milliseconds and the number of timed launches (host arrays of
 * GS_NUM_STAGES). */
gs_status gs_set_profiling(gs_ctx *ctx, int profiling);
gs_status gs_profile_read(gs_ctx *ctx, double *ms, int64_t *count);

/* Default configurations (host structs): 16x16 tiles, batch 32, bg 0,
 * near 0.2, alpha in [1/255, 0.99], T_eps 1e-4, dilation 0.3; Adam
 * beta = (0.9, 0.999), eps 1e-15, lr means 1.6e-4, log-scales 5e-3,
 * quats 1e-3, opacity 5e-2, SH DC 2.5e-3, SH rest 1.25e-4, zero_grads 0. */
gs_status gs_raster_cfg_default(gs_raster_cfg *cfg);
gs_status gs_adam_cfg_default(gs_adam_cfg *cfg);

/* Forward pass (Eq. 2-5 projection, tile binning with per-tile depth sort,
 * Eq. 11 front-to-back compositing; Sec. III-B.3).  Writes colour [3, H, W],
 * depth [H, W] (sum z_i w_i, camera z of the means) and alpha [H, W]
 * (1 - final transmittance).  Any of the three outputs may be NULL.  Keeps
 * the per-pixel final transmittance and last-contributor index, the
 * projected features and the sorted per-tile lists in the context for
 * gs_render_bwd; they stay valid until the next forward call on the context. */
gs_status gs_render_fwd(gs_ctx *ctx, const gs_gaussians *g, const gs_camera *cam,
                        const gs_viewmat *view, const gs_raster_cfg *cfg,
                        float *color, float *depth, float *alpha, gs_stream_t stream);

/* Backward pass of the forward state the context holds: the most recent
 * gs_render_fwd (or batched forward, or training step) on this context.  That
 * state must have been computed from the same Gaussian arrays (the same five
 * pointers, n and SH degree), byte-identical cameras, poses and raster
 * configuration; anything else returns GS_ERR_STATE with nothing enqueued
 * (e.g. two renders at two poses followed by the backward pass of the first).
 * The parameter VALUES are not compared: changing them in place between the
 * forward and the backward pass is the caller's error.  Walks every tile list back to
 * front from the stored last contributor, recomputing transmittance from the
 * stored final T.  dL_dcolor [3, H, W] and dL_ddepth [H, W] are required,
 * dL_dalpha [H, W] may be NULL.  Gradients w.r.t. every parameter array are
 * ADDED to `grads` (the caller zeroes them).  dL_dpose (device float[6],
 * nullable) receives += the gradient w.r.t. xi = (rho, phi) of the left
 * perturbation T_CW(xi) = exp(xi^) T_CW at xi = 0. */
gs_status gs_render_bwd(gs_ctx *ctx, const gs_gaussians *g, const gs_camera *cam,
                        const gs_viewmat *view, const gs_raster_cfg *cfg,
                        const float *dL_dcolor, const float *dL_ddepth, const float *dL_dalpha,
                        const gs_grads *grads, float *dL_dpose, gs_stream_t stream);

/* Token of the forward state the context holds (0 = none): distinct for
 * every forward pass on the context, so a caller that keeps the token of its
 * own forward pass can tell whether the state is still its own before calling
 * a backward pass (and re-run its forward pass if not). */
gs_status gs_state_token(const gs_ctx *ctx, uint64_t *token);

/* One single-view optimisation iteration's backward half (Sec. III-B.3:
 * each iteration optimises the map on one frame): the backward pass of the
 * most recent gs_render_fwd fused with the Adam step.  Computes exactly
 * gs_render_bwd into zeroed gradients followed by gs_adam_step, but never
 * writes the parameter gradients: each Gaussian's gradient is applied by the
 * thread that computes it.  `params` is the flat parameter buffer (layout
 * above) that `g` must point into; m, v are the Adam moments (same layout).
 * step >= 1 is the Adam step; step = 0 instead increments the context's
 * device-side step counter and uses it (no host value changes between
 * calls, so a captured CUDA graph can replay the call; see
 * gs_ctx_set_adam_step).  cfg->zero_grads is ignored.  dL_dpose as in
 * gs_render_bwd. */
gs_status gs_render_bwd_adam(gs_ctx *ctx, const gs_gaussians *g, const gs_camera *cam,
                             const gs_viewmat *view, const gs_raster_cfg *cfg,
                             const float *dL_dcolor, const float *dL_ddepth, const float *dL_dalpha,
                             float *params, float *m, float *v, const gs_adam_cfg *adam, int64_t step,
                             float *dL_dpose, gs_stream_t stream);

/* ---------------------------------------------------------------------------
 * Batched multi-view form.  One call renders, differentiates or scores
 * n_views in [1, GS_MAX_VIEWS] views of one Gaussian map, each with its own
 * camera, pose and image size.  The paper runs its per-frame iterations one
 * view at a time (Sec. III-B.3 optimises on the current frame, keyframes are
 * revisited in later iterations); the batched calls compute the same
 * quantities for all views in one pass over the map, with each kernel
 * launched once for the whole batch (the tiles of all views form one grid).
 * Per-view arguments are HOST arrays of length n_views: cams, views and the
 * image pointer arrays (whose entries are device pointers to that view's
 * images, sized by its camera).  The batched loss is the sum over views of
 * the per-view loss of gs_loss_l1 (each normalised by its own pixel count),
 * so its gradient w.r.t. the map is the sum of the per-view gradients, and a
 * batched step applies one Adam update to that sum.  Limits: n_views * n <
 * 2^31 and fewer than 2^31 pixels and tiles over the batch.
 * ------------------------------------------------------------------------- */
#define GS_MAX_VIEWS 16

/* gs_render_fwd for n_views views.  color, depth, alpha: host arrays of
 * n_views device pointers (each array nullable, each entry nullable).  The
 * state for gs_render_bwd_batched / gs_render_bwd_adam_batched stays in the
 * context as for gs_render_fwd. */
gs_status gs_render_fwd_batched(gs_ctx *ctx, const gs_gaussians *g, int32_t n_views,
                                const gs_camera *cams, const gs_viewmat *views, const gs_raster_cfg *cfg,
                                float *const *color, float *const *depth, float *const *alpha,
                                gs_stream_t stream);

/* gs_render_bwd for the views of the most recent gs_render_fwd_batched (same
 * g, n_views, cams, views, cfg; GS_ERR_STATE otherwise).  dL_dcolor,
 * dL_ddepth: host arrays of n_views device pointers (required); dL_dalpha:
 * nullable array, nullable entries.  The parameter gradients summed over the
 * views are ADDED to grads.  dL_dpose (device float[n_views][6], nullable)
 * receives += each view's pose-twist gradient. */
gs_status gs_render_bwd_batched(gs_ctx *ctx, const gs_gaussians *g, int32_t n_views,
                                const gs_camera *cams, const gs_viewmat *views, const gs_raster_cfg *cfg,
                                const float *const *dL_dcolor, const float *const *dL_ddepth,
                                const float *const *dL_dalpha, const gs_grads *grads, float *dL_dpose,
                                gs_stream_t stream);

/* gs_render_bwd_adam for a batch: the backward pass of the most recent
 * gs_render_fwd_batched fused with ONE Adam step on the gradient summed over
 * the views.  Same arguments and step / device-counter rules as
 * gs_render_bwd_adam, per-view arrays as in gs_render_bwd_batched. */
gs_status gs_render_bwd_adam_batched(gs_ctx *ctx, const gs_gaussians *g, int32_t n_views,
                                     const gs_camera *cams, const gs_viewmat *views, const gs_raster_cfg *cfg,
                                     const float *const *dL_dcolor, const float *const *dL_ddepth,
                                     const float *const *dL_dalpha, float *params, float *m, float *v,
                                     const gs_adam_cfg *adam, int64_t step, float *dL_dpose,
                                     gs_stream_t stream);

/* gs_loss_l1 summed over n_views views: loss (device float[1]) = sum over v of
 * L_v, where L_v is gs_loss_l1's loss of view v; writes every view's
 * dL/dcolor and dL/ddepth.  All image arguments are host arrays of n_views
 * device pointers (none NULL). */
gs_status gs_loss_l1_batched(gs_ctx *ctx, int32_t n_views, const gs_camera *cams,
                             const float *const *color, const float *const *depth,
                             const float *const *target_rgb, const float *const *target_depth,
                             float w_color, float w_depth, float *loss, float *const *dL_dcolor,
                             float *const *dL_ddepth, gs_stream_t stream);

/* One optimisation iteration of the online optimisation (Sec. III-B.3) in
 * one call: the forward pass with the loss of gs_loss_l1 (Eq. 12 plus the
 * depth term) computed in the compositing epilogue, then the backward pass
 * fused with the Adam step, as gs_render_bwd_adam.  The same result as
 * gs_render_fwd + gs_loss_l1 + gs_render_bwd_adam (the same image
 * gradients; the loss value is summed in another order), but the rendered
 * images and the loss image gradients never go to caller memory: the
 * context keeps the gradients.  target_rgb [3, H, W], target_depth [H, W]
 * (0 = invalid); loss (device float[1]) receives L; params / m / v, adam and
 * step as in gs_render_bwd_adam (step = 0: device step counter).  The
 * forward state stays in the context as after gs_render_fwd. */
gs_status gs_train_step(gs_ctx *ctx, const gs_gaussians *g, const gs_camera *cam, const gs_viewmat *view,
                        const gs_raster_cfg *cfg, const float *target_rgb, const float *target_depth,
                        float w_color, float w_depth, float *loss, float *params, float *m, float *v,
                        const gs_adam_cfg *adam, int64_t step, gs_stream_t stream);

/* gs_train_step for a batch of views: loss = sum over views of L_v, one Adam
 * step on the summed gradient (as gs_loss_l1_batched and
 * gs_render_bwd_adam_batched).  target_rgb, target_depth: host arrays of
 * n_views device pointers; color, depth, alpha: optional host arrays of
 * n_views device pointers (each array and entry nullable) that receive the
 * rendered images. */
gs_status gs_train_step_batched(gs_ctx *ctx, const gs_gaussians *g, int32_t n_views, const gs_camera *cams,
                                const gs_viewmat *views, const gs_raster_cfg *cfg,
                                const float *const *target_rgb, const float *const *target_depth,
                                float w_color, float w_depth, float *loss, float *params, float *m, float *v,
                                const gs_adam_cfg *adam, int64_t step, float *const *color,
                                float *const *depth, float *const *alpha, gs_stream_t stream);

/* Tile-shape autotuner (no counterpart in the paper, whose rasterizer uses
 * one fixed tile size).  Times, for each of the GS_AUTOTUNE_CANDIDATES tile
 * shapes 16x16, 8x32 and 32x8 (in that order), `reps` passes of everything
 * the tile shape changes -- the batched forward pass (projection, binning,
 * per-tile sort, compositing) and the raster backward pass -- on the given
 * map and views (n_views >= 1; a single view is n_views = 1), and writes the
 * fastest shape to cfg->tile_w / cfg->tile_h (the other cfg fields are used
 * as given).  ms (host float[GS_AUTOTUNE_CANDIDATES], nullable) receives the
 * milliseconds per pass of each candidate.  The result does not depend on the
 * tile shape (a Gaussian takes part in a pixel by its own support rule), so
 * only speed is compared.  Synchronises; the context's forward state is
 * cleared (run gs_render_fwd again before a backward pass); the list entries a
 * warp stages per round are fixed at 32 (one per lane) and not searched. */
#define GS_AUTOTUNE_CANDIDATES 3
gs_status gs_autotune(gs_ctx *ctx, const gs_gaussians *g, int32_t n_views, const gs_camera *cams,
                      const gs_viewmat *views, gs_raster_cfg *cfg, int32_t reps, float *ms,
                      gs_stream_t stream);

/* Photometric loss (Eq. 12) plus a depth term:
 *   L = w_color * mean over 3HW of |color - target_rgb|
 *     + w_depth * mean over pixels with target_depth > 0 of |depth - target_depth|.
 * Writes L to loss (device float[1]) and dL/dcolor, dL/ddepth (sign(0) = 0). */
gs_status gs_loss_l1(gs_ctx *ctx, const gs_camera *cam, const float *color, const float *depth,
                     const float *target_rgb, const float *target_depth, float w_color, float w_depth,
                     float *loss, float *dL_dcolor, float *dL_ddepth, gs_stream_t stream);

/* Largest image gs_loss_l1_noalloc accepts: 2^24 pixels (e.g. 4096 x 4096). */
#define GS_LOSS_NOALLOC_MAX_PIXELS (1 << 24)

/* gs_loss_l1 without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory,
 * such as a process whose GPU memory all belongs to its own pool (a raw
 * cudaMalloc would fail or fragment it) or a latency-critical loop that cannot
 * absorb an allocation and the synchronisation it implies.  Same arguments
 * (minus the context), outputs and results as gs_loss_l1.  It runs on the
 * calling thread's current CUDA device and takes its scratch from a fixed
 * array compiled into the library (about 96 KB on every GPU that loads the
 * library, held until the process exits); it calls no cudaMalloc/cudaFree.
 * - Images larger than GS_LOSS_NOALLOC_MAX_PIXELS pixels are rejected with
 *   GS_ERR_CAPACITY before anything is enqueued.
 * - The first call on a device looks up that device's address of the array;
 *   make this first call before any stream capture on that device.
 * - Every call on a device uses the same array: calls whose kernels may
 *   overlap on the GPU (different streams with no ordering between them)
 *   race and give wrong results.  Calls ordered on one stream are safe, since
 *   each call writes every scratch value before it reads it. */
gs_status gs_loss_l1_noalloc(const gs_camera *cam, const float *color, const float *depth,
                             const float *target_rgb, const float *target_depth, float w_color, float w_depth,
                             float *loss, float *dL_dcolor, float *dL_ddepth, gs_stream_t stream);

/* One dense Adam step over the flat parameter buffer (layout above):
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   p -= lr_group * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * The paper optimises "using the gradient descent method" (Sec. III-B.3);
 * Adam is the optimiser used here.  step >= 1 is the Adam step; step = 0
 * instead increments the context's device-side step counter and uses it
 * (as gs_render_bwd_adam does; graph-capturable).  params, m, v updated in
 * place; grads read, and cleared to 0 when cfg->zero_grads is 1 (ready for
 * the next accumulating gs_render_bwd). */
gs_status gs_adam_step(gs_ctx *ctx, float *params, float *grads, float *m, float *v,
                       int64_t n, int32_t sh_degree, const gs_adam_cfg *cfg, int64_t step,
                       gs_stream_t stream);

/* The tile-binning stage on its own (Sec. III-B.3: tiles, per-tile depth
 * order), for exact checks: per Gaussian mean2d [n, 2], support half-extents
 * extent [n, 2] (a Gaussian takes part iff both are > 0) and depth [n] (> 0).
 * With tw, th powers of two, TX = ceil(W / tw), TY = ceil(H / th) and float32
 * arithmetic, a Gaussian covers tiles [x0, x1) x [y0, y1),
 *   x0 = clamp(floor((mx - ex) / tw), 0, TX), x1 = clamp(floor((mx + ex) / tw) + 1, 0, TX).
 * Outputs: keys [P] = (tile << 32) | bits(depth), ids [P] sorted by key with
 * ties in index order, ranges [TX * TY, 2] = [first, last + 1) per tile
 * ((0, 0) if empty), *n_pairs (host) = P.  Returns GS_ERR_CAPACITY (and sets
 * *n_pairs) if P > pair_capacity (keys/ids then untouched).  Synchronises. */
gs_status gs_bin_tiles(gs_ctx *ctx, int64_t n, const float *mean2d, const float *extent,
                       const float *depth, int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                       uint64_t *keys, uint32_t *ids, uint32_t *ranges, int64_t pair_capacity,
                       int64_t *n_pairs, gs_stream_t stream);

/* Per-frame seeding of new Gaussians (Sec. III-B.2, Eq. 10) on the device.
 * The frame rgb [3, H, W] (values in [0, 1]) is covered by a grid of square
 * root cells of max_size px (clipped at the border); a cell splits into its
 * four (clipped, non-empty) quadrants while the mean over the three channels
 * of the per-channel pixel variance exceeds var_thr (0.01: the paper's
 * contrast threshold 0.1 read as a standard deviation), its side exceeds
 * min_size and it holds more than one pixel; cells that do not split are
 * leaves.  max_size and min_size are powers of two, 1 <= min <= max <= 4096.
 *
 * gs_quadtree_leaves writes the leaves as int32 (x0, y0, w, h) rows to
 * `leaves` (device [capacity, 4], in no particular order) and their number to
 * *n_leaves (host); GS_ERR_CAPACITY if they do not fit.  Synchronises. */
gs_status gs_quadtree_leaves(gs_ctx *ctx, const float *rgb, int32_t width, int32_t height, float var_thr,
                             int32_t max_size, int32_t min_size, int32_t *leaves, int64_t capacity,
                             int64_t *n_leaves, gs_stream_t stream);

/* gs_seed_quadtree: the quadtree of the frame (size from cam), then one new
 * Gaussian per leaf whose centre pixel (min(floor(x0 + w/2), W - 1),
 * min(floor(y0 + h/2), H - 1)) has depth > 0 and, if alpha (the rendered
 * alpha image [H, W] of the current map, nullable) is given, alpha <
 * alpha_thr (the novelty rule, 0.5).  Eq. 10 back-projects the leaf centre u
 * with that depth z: p_w = R^T (((u_x - cx) z / fx, (u_y - cy) z / fy, z) - t)
 * (float32, evaluated left to right, R^T's products summed in row order);
 * log-scales log(sqrt(w^2 + h^2) / 2 * z / fx) on all axes, quaternion
 * (1, 0, 0, 0), opacity logit 0, SH DC (c - 0.5) / Y_00 from the pixel colour
 * c, higher bands 0.  The parameters go to rows [0, k) of the caller's arrays
 * (device, each with `capacity` rows in the layout of gs_gaussians, e.g. the
 * free slots of a map), in no particular order; *n_seeded (host) = k.  If
 * k > capacity only `capacity` rows are written and GS_ERR_CAPACITY is
 * returned with *n_seeded = k.  Synchronises (twice). */
gs_status gs_seed_quadtree(gs_ctx *ctx, const float *rgb, const float *depth, const float *alpha, float alpha_thr,
                           const gs_camera *cam, const gs_viewmat *view, int32_t sh_degree, float var_thr,
                           int32_t max_size, int32_t min_size, float *means, float *log_scales, float *quats,
                           float *opacity_logits, float *sh, int64_t capacity, int64_t *n_seeded,
                           gs_stream_t stream);

/* ---------------------------------------------------------------------------
 * TSDF fusion (Sec. III-B.1, Eq. 6-9) and the voxel-weight novelty check of
 * the per-frame seeding (Sec. III-B.2).
 *
 * The grid is single resolution: voxels of side voxel_size in blocks of 8^3,
 * found through an open-addressing hash table of table_size buckets over a
 * pool of `capacity` block slots.  Every array is device memory owned by the
 * caller and set once before the first call: keys all 0xFF bytes (free
 * buckets), stamps 0, voxels 0, claims all 0xFF bytes, counters 0; slots and
 * touched need no initial value.  Block (bx, by, bz), each coordinate in
 * [-2^20, 2^20), has the key ((bx + 2^20) << 42) | ((by + 2^20) << 21) |
 * (bz + 2^20); voxel (x, y, z) of the block (0..7 each) holds its tsdf and
 * weight at voxels[2 (512 slot + x + 8 y + 64 z)] and [... + 1], and its
 * centre is at (8 b + (x, y, z) + 0.5) voxel_size in the world frame.
 * ------------------------------------------------------------------------- */
#define GS_TSDF_BLOCK 8
#define GS_TSDF_MAX_SAMPLES 16

typedef struct {
  uint64_t *keys;     /* [table_size] block keys; all-ones = free */
  int32_t *slots;     /* [table_size] pool slot of each bucket's block */
  uint32_t *stamps;   /* [table_size] id of the last frame that touched the bucket */
  float *voxels;      /* [capacity, 512, 2] (tsdf, weight) */
  uint32_t *claims;   /* [capacity, 512] seeding scratch, all 0xFFFFFFFF between calls */
  uint32_t *touched;  /* [table_size / 2] buckets touched by the last allocation */
  uint32_t *counters; /* [4]: slots handed out (may exceed capacity), buckets touched by the
                         last allocation, failed inserts, voxels updated (accumulates) */
  int64_t table_size; /* power of two in [2, 2^32] */
  int64_t capacity;   /* pool slots in [1, 2^31 - 1] */
  float voxel_size;   /* s (metres) */
  float truncation;   /* eps (metres); at most GS_TSDF_MAX_SAMPLES band samples: eps <= 30 s */
  float max_weight;   /* w_max >= 1 (Eq. 8) */
  int32_t fusion;     /* 0: Eq. 9 as printed, the new tsdf weighted by w_k;
                         1: weighted by 1 (KinectFusion's running average) */
} gs_tsdf_grid;

/* gs_tsdf_integrate: fuse the depth image [H, W] (camera z in metres, <= 0 =
 * no measurement; size from cam) seen with the world-to-camera pose `view`.
 * Allocation: the ray through every pixel centre (i + 0.5, j + 0.5) with
 * depth D > 0 is sampled at camera depths D - eps + k 2 eps / n, k = 0..n,
 * n = ceil(eps / 2s) (samples at z <= 0 dropped); each block holding a sample
 * is inserted (a new key takes the next slot, counters[0]++) and listed once
 * in `touched` (stamps[bucket] = frame).  Integration (Eq. 6-9), for every
 * voxel of the touched blocks: p_c = R p_v + t; skipped if z <= 0, if the
 * projection (fx x/z + cx, fy y/z + cy) is outside the image, if the depth
 * at its pixel (floor of the projection) is not > 0, or if sdf = D - z <
 * -eps; otherwise tsdf = clamp(sdf / eps, -1, 1), w_k = min(w_max, w_{k-1} +
 * 1) and the average of `fusion`.  The block, pixel and update decisions are
 * float32 with correctly rounded operations in the order written here.
 * `frame` (>= 1) must differ from the previous call's.  The table must have
 * room: with table_size >= 2 (blocks + W H (n + 1)) no insert can fail;
 * failures are counted in counters[2] and their blocks skipped.  Blocks whose
 * slot is >= capacity are skipped too: after the caller grows the pool,
 * min_slot = the old capacity re-runs only the integration, over the last
 * touched list, for the slots >= min_slot (same depth, camera and pose).
 * min_slot = 0 runs both steps.  Asynchronous; gs_tsdf_counters reads the
 * counters. */
gs_status gs_tsdf_integrate(gs_ctx *ctx, const gs_tsdf_grid *grid, const float *depth, const gs_camera *cam,
                            const gs_viewmat *view, uint32_t frame, int64_t min_slot, gs_stream_t stream);

/* Synchronise the stream and copy the 4 counters to out (host).  Returns
 * GS_ERR_CAPACITY if counters[0] > capacity (grow the pool, then
 * gs_tsdf_integrate with min_slot) or counters[2] > 0 (table too small). */
gs_status gs_tsdf_counters(gs_ctx *ctx, const gs_tsdf_grid *grid, int64_t *out, gs_stream_t stream);

/* Insert every key of `from` into `to` (same pool: the slot of each key is
 * kept; to's keys all free, to.table_size a power of two > from's count of
 * keys).  Between frames only: the touched list refers to buckets of `from`. */
gs_status gs_tsdf_rehash(gs_ctx *ctx, const gs_tsdf_grid *from, const gs_tsdf_grid *to, gs_stream_t stream);

/* tsdf[i], weight[i] (each nullable) of the voxel holding world point
 * points[i] (float [n, 3]; voxel floor(p / s), float32 division), 0 and 0 where its
 * block is not allocated. */
gs_status gs_tsdf_query(gs_ctx *ctx, const gs_tsdf_grid *grid, const float *points, int64_t n, float *tsdf,
                        float *weight, gs_stream_t stream);

/* gs_seed_tsdf: gs_seed_quadtree with the paper's novelty check instead of
 * the rendered alpha.  After gs_tsdf_integrate of this frame, a leaf seeds
 * iff the voxel holding its Eq. 10 point (p_w in float32, correctly rounded
 * operations in the order of gs_seed_quadtree's formula, voxel floor(p_w /
 * s) with a float32 division) has weight exactly 1, and at most one leaf
 * seeds each voxel: the one with the smallest y0 W + x0.  Means are that
 * p_w; the other parameters as in gs_seed_quadtree.  Synchronises (twice). */
gs_status gs_seed_tsdf(gs_ctx *ctx, const float *rgb, const float *depth, const gs_tsdf_grid *grid,
                       const gs_camera *cam, const gs_viewmat *view, int32_t sh_degree, float var_thr,
                       int32_t max_size, int32_t min_size, float *means, float *log_scales, float *quats,
                       float *opacity_logits, float *sh, int64_t capacity, int64_t *n_seeded, gs_stream_t stream);

/* Failure detection.  gs_count_nonfinite: *count (host) = the number of
 * NaN / +-Inf floats in the device array x[0, n) (e.g. a map's flat
 * parameters after a step); returns GS_ERR_NONFINITE if any.  Synchronises.
 * gs_ctx_inject_alloc_failure: the after-th next growth of the context's
 * scratch (1 = the next one; 0 disarms) fails with GS_ERR_OOM before any
 * buffer is touched, so callers can test their recovery; the context stays
 * usable (a real allocation failure part-way through a growth drops that
 * scratch group, which the next call allocates again). */
gs_status gs_count_nonfinite(gs_ctx *ctx, const float *x, int64_t n, int64_t *count, gs_stream_t stream);
gs_status gs_ctx_inject_alloc_failure(gs_ctx *ctx, int32_t after);

/* Bounds-checked build (libgsplat_checked.so, compiled with GS_CHECKED; no
 * counterpart in the paper: the stand-in for a race / memory checker).  Its
 * kernels check every index they read from memory (list ids against the
 * projected records, tile ranges against the pair buffer, tile numbers
 * against the grid, ids against the items in the per-tile sort) before using
 * it; a violation sets the context's bounds word and the access is skipped or
 * redirected to a valid dummy (never a trap), and the next gs_sync_status
 * returns GS_ERR_BOUNDS and clears the word.  The word's address is bound
 * per library at context creation (the newest context's word collects the
 * violations of all contexts of the process).  Results are otherwise those
 * of the normal build.  gs_bounds_checked: 1 in the checked build, 0 in the
 * normal one (no device access).  gs_ctx_inject_bounds_fault: sets the bounds
 * word from the host, as a violation would, so callers can test the
 * reporting path without a device fault; synchronises. */
int gs_bounds_checked(void);
gs_status gs_ctx_inject_bounds_fault(gs_ctx *ctx);

/* Measured issue rates of the two ALU pipes the raster passes run on (no
 * counterpart in the paper: they are the denominators of the raster passes'
 * ALU roofline).  On device `device`, a fully occupied grid runs eight
 * independent chains per thread of FP32 FMA (iters x 128 per thread) and
 * then of MUFU ex2.approx (iters / 4 x 128 per thread), each timed with CUDA
 * events after a warm-up launch; one thread reads the SM cycle counter and
 * the global timer around its loop, which gives the SM clock of the run.
 * iters in [1, 2^24]; about 50 ms per probe at iters = 50000 on a GB300.
 * Synchronises the device; allocates 36 bytes of device memory for the run. */
typedef struct {
  double fma_tflops;     /* 2 flop per FMA lane-instruction, whole GPU, TFLOP/s */
  double ex2_gops;       /* ex2 lane-results per second, whole GPU, G/s */
  double fma_sm_mhz;     /* SM clock during the FMA probe */
  double ex2_sm_mhz;     /* SM clock during the ex2 probe */
  double fma_per_sm_clk; /* FMA lane-instructions per SM per clock */
  double ex2_per_sm_clk; /* ex2 lane-results per SM per clock */
  double fma_ms, ex2_ms; /* event time of each timed launch */
  int32_t num_sms;       /* multiprocessors of the device */
} gs_alu_peaks;
gs_status gs_measure_alu_peaks(int device, int32_t iters, gs_alu_peaks *out);

/* Copy the last forward pass's projected per-Gaussian quantities to caller
 * buffers (each nullable), n = views x Gaussians items, item v * N + i being
 * Gaussian i seen from view v: mean2d [n, 2] (high part of a double-float),
 * cov2d [n, 3] (a, b, c of the dilated 2D covariance [[a, b], [b, c]]),
 * depth [n], rgb [n, 3], opacity [n], tiles [n] (int32 tiles touched; 0 =
 * culled).  For parity checks of the projection step. */
gs_status gs_get_projection(gs_ctx *ctx, float *mean2d, float *cov2d, float *depth, float *rgb,
                            float *opacity, int32_t *tiles, gs_stream_t stream);

/* Copy the last forward pass's per-tile list ranges to `ranges` (device
 * uint32 [n_tiles, 2]: [first, last + 1) into the depth-sorted pair list,
 * (0, 0) for an empty tile); n_tiles must be the forward pass's tile count
 * (the views' tiles end to end, row-major within a view).  For parity checks
 * of the binning and for picking the longest-list tiles. */
gs_status gs_get_tile_ranges(gs_ctx *ctx, uint32_t *ranges, int64_t n_tiles, gs_stream_t stream);

/* Copy the raster visit order of the last forward pass to `order` (device
 * uint32 [n_tiles], a permutation of the tiles numbered as in
 * gs_get_tile_ranges, their length classes non-increasing: class 0 for an
 * empty list, else 4 floor(log2 len) + the two bits after len's leading one
 * + 1); n_tiles must be the forward pass's tile count.  GS_ERR_STATE when
 * that pass visited the tiles in index order (gs_ctx_set_tile_order(0), or
 * the radix binning of very long lists).  For checks of the binning. */
gs_status gs_get_tile_order(gs_ctx *ctx, uint32_t *order, int64_t n_tiles, gs_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GSPLAT_H */
