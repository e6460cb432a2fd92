/*
 * splatloam.h -- C ABI of libsplatloam, a GB300 (sm_103a) differentiable rasterizer of 2D
 * Gaussian primitives into LiDAR spherical range images, after Splat-LOAM (arXiv 2503.17491).
 *
 * What the library computes (the paper's statement of the problem):
 *   render   : primitives {o, mu, R = (t_alpha, t_beta, t_n), s} (Sec. 3.2, Eq. world_T_splat),
 *              a sensor pose and LiDAR intrinsics -> per-pixel range D, normal N and accumulated
 *              opacity O by front-to-back alpha blending over per-tile lists sorted by range
 *              (Sec. 3.2.1, Eqs. ab_depth, ab_normal, ab_opacity), each ray intersected with each
 *              splat as two planes (Sec. 3.2.2, Eq. planes_to_splat; Supp. D.1), with a spherical
 *              bounding box that handles the +-pi azimuth seam (Sec. 3.2.3, Supp. B).
 *   backward : per-pixel dL/dD, dL/dN, dL/dO -> dL/d(every primitive parameter) (Supp. D.2, with
 *              the dL/dO channel and the chain rule through the parametrisation below).
 *   loss     : L_d + lambda_n L_n (+ lambda_o L_o) over valid pixels (Sec. 3.3.2, Eqs.
 *              loss_range, loss_normal, loss_opacity), with its per-pixel gradients.
 *   adam     : one Adam step of all primitive parameters (the paper does not name its
 *              optimiser; Adam is used here).
 *
 * Conventions (every call):
 *   - Primitive parameters, one row per primitive, float32, device memory owned by the caller:
 *       pos_logit  n x 4 : (mu_x, mu_y, mu_z, logit(o))       o = 1 / (1 + exp(-logit))
 *       quat_wxyz  n x 4 : (w, x, y, z), any nonzero length   R = R(q / |q|), columns t_a, t_b, t_n
 *       log_scale  n x 2 : (log s_alpha, log s_beta)          s = exp(log_scale)
 *   - Poses: T_world_sensor is a host array of 16 doubles, row-major 4x4, sensor -> world, a
 *     rigid transform.  The library inverts it in FP64 to get T^c_w (Sec. 3.2.2).
 *   - Sensor frame: x forward, y left, z up (Sec. 3.1).  Pixel (r, c) of a rows x cols image
 *     looks along azimuth pi - 2 pi (c + 1/2) / cols and elevation
 *     elev_max - r (elev_max - elev_min) / (rows - 1); column cols/2 - 1/2 looks along +x.
 *   - Images: all registered views are packed one after the other.  View v occupies pixels
 *     [pixel_offset(v), pixel_offset(v) + rows_v * cols_v) of a buffer of P = sum rows_v cols_v
 *     pixels, row-major inside the view.  depth and alpha are float32[P]; normal is float32[3][P]
 *     (three planes of P pixels: x, y, z).  N is in the sensor frame of its view; D is the blended
 *     range (not divided by O).
 *   - Every compute call is asynchronous and stream-ordered on `stream` (a cudaStream_t, or NULL
 *     for the legacy default stream), never synchronises the host and never allocates: all
 *     workspace is owned by the context and sized at creation, so a sequence of calls can be
 *     captured into a CUDA graph.  Exceptions: splat_ctx_create/destroy, splat_set_views (which
 *     uploads view tables synchronously) and splat_get_status/splat_get_stats/splat_debug_copy
 *     (which synchronise).
 *   - Return codes: SPLAT_OK, or an error code (errors never cross the ABI as exceptions).
 *     Errors found on the device (capacity overflow, non-finite input) are recorded in a status
 *     word and reported by splat_get_status after the stream is synchronised.
 *   - A context is not thread-safe; use one per host thread / stream.
 */
#ifndef SPLATLOAM_H
#define SPLATLOAM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPLAT_API __attribute__((visibility("default")))

typedef struct splat_ctx splat_ctx;

/* Return codes. */
enum {
    SPLAT_OK = 0,
    SPLAT_ERR_INVALID_ARG = 1,  /* null pointer, bad size, non-finite pose, rows/cols < 2, ... */
    SPLAT_ERR_CUDA = 2,         /* a CUDA runtime call failed; see splat_last_cuda_error       */
    SPLAT_ERR_CAPACITY = 3,     /* more (tile, primitive) pairs than max_pairs: outputs invalid */
    SPLAT_ERR_TIMEOUT = 4,      /* a bounded device wait gave up                               */
    SPLAT_ERR_NONFINITE = 5,    /* a primitive had a non-finite value or a zero quaternion     */
    SPLAT_ERR_STATE = 6,        /* call order violated (e.g. backward before any render)       */
    SPLAT_ERR_UNSUPPORTED = 7   /* configuration not built into this library (tile shape)      */
};

/* Bits of the device status word (splat_get_status). */
enum {
    SPLAT_STATUS_CAPACITY = 1u,
    SPLAT_STATUS_NONFINITE = 2u,
    SPLAT_STATUS_TIMEOUT = 4u
};

/* LiDAR intrinsics of one view: image size and elevation range in radians
 * (elev_min < elev_max, both inside (-pi/2, pi/2)); azimuth always spans 360 degrees. */
typedef struct {
    int32_t rows, cols;
    float elev_min, elev_max;
} splat_lidar_intrinsics;

/* The primitives (device pointers, caller-owned; layout in the header comment). */
typedef struct {
    const float *pos_logit;   /* n x 4 */
    const float *quat_wxyz;   /* n x 4 */
    const float *log_scale;   /* n x 2 */
    int64_t n;
} splat_gaussians;

/* Rasterizer settings.  The paper gives no cutoffs; the defaults are the 3DGS conventions it
 * builds on (Sec. 3.2.1): alpha_min 1/255, alpha_max 0.99, t_min 1e-4, plus the 3-sigma box of
 * Sec. 3.2.3 (sigma_cut 3).  Tiles are tile_h x tile_w pixels with tile_h * tile_w == 256;
 * built shapes: 16x16 (the paper's), 8x32, 32x8, 4x64.  flip_normals = 1 turns each normal
 * towards the sensor.  work_cap is reserved (must be 0). */
typedef struct {
    float alpha_min, alpha_max, t_min, sigma_cut;
    int32_t tile_h, tile_w, work_cap, flip_normals;
} splat_render_config;

/* Workspace limits fixed at creation.  max_pairs bounds the number of (tile, primitive) pairs
 * of one render call summed over views; max_tiles = 0 derives a bound from max_pixels. */
typedef struct {
    int64_t max_gaussians;
    int32_t max_views;
    int64_t max_pixels;
    int64_t max_pairs;
    int64_t max_tiles;
} splat_capacity;

/* Loss weights of Eq. loss_full: o_eps floors O inside -log O; rho_d of Eq. loss_range, a
 * weight that depends on the measured range and has no printed form, is read as Dt^rho_exp.
 * lambda_s and tau_s weigh the scale term of splat_refine_step, lambda_s sum_i max(0,
 * max(s_a, s_b)_i - tau_s) (the penalty of Eq. L_s with its sign read as growth beyond tau_s; 0
 * disables it).
 * normal_mode selects the normal term of Eq. loss_normal:
 *   SPLAT_NORMALS_TARGET (0): lambda_n (1 - N(u) . Nt(u)) against the target normals;
 *   SPLAT_NORMALS_RANGE_MAP (1): self-regularised, lambda_n (1 - N(u) . n_D(u)) with n_D the
 *     normal of the rendered range map D (after 2DGS): for u = (r, c), r + 1 < rows,
 *     x = (r, c + 1 mod cols), y = (r + 1, c), P(w) = D(w) v(w) (v the pixel-centre ray),
 *     m = (P(x) - P(u)) x (P(y) - P(u)), n_D = -sign(m . v(u)) m / |m| (facing the sensor),
 *     counted where the targets of u, x and y are valid, D > 0 at all three and m != 0 (a zero
 *     range puts P at the sensor, where the side is undefined; the sign is held fixed in the
 *     gradient, which reaches D at u, x and y).  Needs the views' geometry: splat_view_loss and
 *     splat_refine_step only; target_normal may be NULL there. */
enum { SPLAT_NORMALS_TARGET = 0, SPLAT_NORMALS_RANGE_MAP = 1 };
typedef struct {
    float lambda_n, lambda_o, o_eps;
    float lambda_s, tau_s;
    int32_t normal_mode;
    float rho_exp;            /* rho_d = target_depth^rho_exp weighs the L1 range term (0: 1) */
} splat_loss_config;

/* Map growth (Sec. 3.3.1 local model initialisation, Sec. 3.3.2 densification).
 *   refine = 0: the mask is M_v (target range > 0); refine = 1: M_v and (M_n or M_e), with
 *     M_n = O <= lambda_do and M_e = |D - Dt| >= lambda_de on the rendered images (binary32).
 *   Weight of a masked pixel from the range gradients of the target: g_x = Dt(r, c + 1 mod W) -
 *     Dt(r, c), g_y = Dt(r + 1, c) - Dt(r, c) (0 where a neighbour is missing or invalid),
 *     w = min((w0 + |g_x|) + |g_y|, w_cap) in binary32, counted as q = floor(256 w).
 *   New primitive of a drawn pixel: centre T_ws (Dt v), normal towards the sensor (the
 *     shortest-arc rotation from e_z to -R_ws v; (0, 1, 0, 0) when that normal is -e_z within
 *     1e-6), log-scales log(scale_k Dt sqrt(dgamma dtheta)) on both axes, opacity `opacity`.
 *   seed: key of the Philox-4x32-10 stream of the draw. */
typedef struct {
    int32_t refine;
    float lambda_do, lambda_de;
    float w0, w_cap;          /* metres; 0 <= w0, 0 < w_cap <= 16 */
    float scale_k, opacity;   /* scale_k > 0, 0 < opacity < 1      */
    uint64_t seed;
} splat_densify_config;

/* Adam settings; one learning rate per parameter group. */
typedef struct {
    float lr_pos, lr_opacity, lr_rot, lr_scale;
    float beta1, beta2, eps;
} splat_adam_config;

/* Counters of the last render / backward call (synchronising). */
typedef struct {
    int64_t n_pairs;          /* (tile, primitive) pairs binned, summed over views  */
    int64_t fwd_evals;        /* pixel x primitive intersection tests in the forward */
    int64_t bwd_evals;        /* the same in the backward                            */
    int64_t n_pixels;         /* pixels of the registered views                      */
    int64_t n_tiles;          /* tiles of the registered views                       */
    int64_t kernel_launches;  /* kernels this context has launched since creation    */
    int64_t n_touching;       /* (view, primitive) pairs that touch at least one tile */
} splat_stats;

/* ---- context ------------------------------------------------------------------------------ */

/* Fill cfg with the defaults above (16x16 tiles). */
SPLAT_API void splat_default_config(splat_render_config *cfg);

/* Create a context on the current CUDA device and allocate its workspace (the only place the
 * library allocates device memory).  *out receives the context.  Errors: INVALID_ARG (bad
 * config or capacity), UNSUPPORTED (tile shape), CUDA (allocation failed). */
SPLAT_API int splat_ctx_create(const splat_render_config *cfg, const splat_capacity *cap,
                               splat_ctx **out);

/* Free the context and its workspace (synchronises the device). NULL is ignored. */
SPLAT_API void splat_ctx_destroy(splat_ctx *ctx);

/* Register the views later calls render: n_views poses T_world_sensor (host, n_views x 16
 * doubles, row-major sensor -> world) and intrinsics (host, n_views).  Computes per-view tables
 * (tile frames and per-pixel ray planes, in FP64) and uploads them synchronously, growing their
 * device allocation when a larger view set needs it; not for use under stream capture.  Errors: INVALID_ARG (n_views out of
 * [1, max_views], non-finite or non-rigid pose, rows/cols outside [2, 32767], bad elevation
 * range, more pixels or tiles than the capacity). */
SPLAT_API int splat_set_views(splat_ctx *ctx, int32_t n_views, const double *T_world_sensor,
                              const splat_lidar_intrinsics *intr);

/* Pixel offset of view v in the packed image buffers (-1 if v is not registered). */
SPLAT_API int64_t splat_view_pixel_offset(const splat_ctx *ctx, int32_t v);

/* ---- render ------------------------------------------------------------------------------- */

/* Render every registered view of the primitives g (g->n <= max_gaussians) into the packed
 * buffers depth[P], normal[3][P], alpha[P] (device, caller-owned).  The per-tile lists,
 * transmittances and contributor counts are kept in the context for the next backward call.
 * Stages: per-primitive projection and spherical bounding box (one pass over all views),
 * range sort, tile binning and sort, per-tile front-to-back compositing (one persistent launch
 * over the tiles of all views).  Errors: INVALID_ARG, STATE (no views), CUDA. */
SPLAT_API int splat_render_views(splat_ctx *ctx, const splat_gaussians *g, float *depth,
                                 float *normal, float *alpha, void *stream);

/* Gradient of L with respect to the parameters of the primitives rendered by the last
 * splat_render_views / splat_render call of ctx, given dL/dD (P), dL/dN (3 x P) and dL/dO (P)
 * in the packed layout (NULL means zero).  Writes g_pos_logit (n x 4: dL/dmu, dL/dlogit),
 * g_quat (n x 4, w.r.t. the unnormalised quaternion) and g_log_scale (n x 2), summed over all
 * views; accumulate = 1 adds to the existing contents instead of overwriting.  The back-to-front
 * pass (Supp. D.2) replays, for each pixel, exactly the contributions the forward composited (the
 * forward records them per 4 x 8 pixel block in the context's workspace), recovers the
 * transmittance by division and sums each primitive's per-pixel terms before one set of atomics
 * per (block, primitive).  g must hold the parameters of that render: the replay stages the
 * primitives the render's projection prepared, and the chain rule is taken at g.
 * Errors: INVALID_ARG, STATE (no render before), CUDA. */
SPLAT_API int splat_render_views_backward(splat_ctx *ctx, const splat_gaussians *g,
                                          const float *dL_ddepth, const float *dL_dnormal,
                                          const float *dL_dalpha, float *g_pos_logit,
                                          float *g_quat, float *g_log_scale, int accumulate,
                                          void *stream);

/* One view: splat_set_views(ctx, 1, T_world_sensor, intr) followed by splat_render_views.  Not
 * for stream capture (the view upload is synchronous). */
SPLAT_API int splat_render(splat_ctx *ctx, const splat_gaussians *g,
                           const double T_world_sensor[16], const splat_lidar_intrinsics *intr,
                           float *depth, float *normal, float *alpha, void *stream);

/* Same as splat_render_views_backward (the views are those of the last render). */
SPLAT_API int splat_render_backward(splat_ctx *ctx, const splat_gaussians *g,
                                    const float *dL_ddepth, const float *dL_dnormal,
                                    const float *dL_dalpha, float *g_pos_logit, float *g_quat,
                                    float *g_log_scale, int accumulate, void *stream);

/* Gradient of the loss of the last backward (splat_render_views_backward, splat_render_backward
 * or splat_refine_step) with respect to each registered view's pose, the tracking variable of
 * Sec. 3.3.  The world-to-sensor transform T^c_w enters the render only through the sensor-frame
 * vectors b_alpha = s_alpha R^c_w t_alpha, b_beta, b_c = R^c_w mu + t^c_w and the normal
 * n = +-R^c_w t_n (Supp. D.1).  For the left perturbation T^c_w <- exp(xi^) T^c_w with
 * xi = (rho, omega) in the sensor frame (rho a translation in metres, omega a rotation vector in
 * radians), g_pose[6 v .. 6 v + 5] = (dL/drho, dL/domega) of view v at xi = 0:
 *   dL/drho = sum_i dL/db_c,i,  dL/domega = sum_i (b_c x dL/db_c + b_alpha x dL/db_alpha +
 *   b_beta x dL/db_beta + n x dL/dn)_i.
 * g_pose: device, caller-owned, n_views x 6 floats.  Stream-ordered copy (graph-capturable).
 * The backward forms these terms only while splat_set_pose_gradient(ctx, 1) is in effect (off
 * by default: map refinement does not need them).
 * Errors: INVALID_ARG (null), STATE (no backward with pose terms since the views were set),
 * CUDA. */
SPLAT_API int splat_set_pose_gradient(splat_ctx *ctx, int enable);
SPLAT_API int splat_pose_gradient(splat_ctx *ctx, float *g_pose, void *stream);

/* Keyframe sampling for refinement (Sec. 3.3: a geometric-distribution scheme that selects the
 * most recent keyframe with probability at least 40 % and older ones progressively less often).
 * With draws > 0, every following render (splat_render_views, splat_refine_step) first draws
 * `draws` keyframes on the device from P(age a) = p (1 - p)^a / Z over the registered views (age
 * 0 = the last registered view; p = p_newest, so P(newest) >= p): draw j of call s takes the
 * first word x of Philox-4x32-10 (counter (j, s, 0, 0), key (seed low, seed high)) and its age is
 * the number of thresholds floor(C_a 2^32) (C the FP64 cumulative law, a < n_views - 1) at or
 * below x.  Views not drawn take no primitives in that call (their images are zero) and their
 * pixels do not enter splat_refine_step's loss.  The call counter s restarts at 0 here;
 * splat_set_views turns sampling off.  draws = 0 turns it off.
 * Errors: INVALID_ARG (draws < 0, p_newest outside (0, 1]), STATE (no views), CUDA. */
SPLAT_API int splat_set_view_sampling(splat_ctx *ctx, int draws, double p_newest, uint64_t seed);

/* The views drawn for the last render (1 = drawn), n_views bytes to host memory (synchronising);
 * all ones when sampling is off.  Errors: INVALID_ARG, STATE (no views), CUDA. */
SPLAT_API int splat_get_active_views(splat_ctx *ctx, uint8_t *flags);

/* Back-projection of rendered range images to a point cloud (Sec. 3.3: the local model is sampled
 * by back-projecting the rasterised range image at its estimated pose, p = T_ws phi^-1(u, d)).
 * depth and alpha: packed images of the context's registered views (as rendered); D is the
 * unnormalised blend, so a pixel's range is d = D / O, taken where O >= o_min (o_min > 0).
 * Writes points (device, caller-owned, 3 x P planar, world frame) from the pixel-centre ray of
 * the spherical projection and the view's pose; NaN where O < o_min.  Stream-ordered.
 * Errors: INVALID_ARG (null, o_min <= 0), STATE (no views), CUDA. */
SPLAT_API int splat_backproject(splat_ctx *ctx, const float *depth, const float *alpha,
                                float o_min, float *points, void *stream);

/* Map growth over the packed pixels of the registered views (Sec. 3.3.1, 3.3.2): the mask and
 * weights of splat_densify_config, then one systematic weighted draw of n_new samples over all
 * packed pixels (Q = sum of the weights q, C_i the exclusive prefix in packed order; sample j
 * sits at s_j = floor((j Q + o) / n_new) and belongs to the pixel with C_i <= s_j < C_i + q_i;
 * o = floor(x Q / 2^32) with x the first word of Philox-4x32-10((0, c, 2, 0), (seed lo, seed
 * hi)), c the number of earlier splat_densify calls on this context).  Slot j of the new
 * primitives, index n_old + j of pos_logit [capacity][4], quat [capacity][4] and log_scale
 * [capacity][2] (device, caller-owned), receives the primitive of the pixel whose first sample
 * is j; a slot whose sample falls on a pixel drawn before it, and every slot when no pixel is
 * masked, is written empty (centre 0, opacity logit -30: below alpha_min, so it takes no pairs
 * and no gradient; identity rotation; log-scales 0).  The caller zeroes the optimiser moments of
 * the new slots.  target_depth [P]; depth and alpha [P] (as rendered) are read when
 * cfg->refine.  Stream-ordered, no synchronisation or allocation (capturable); uses the
 * context's gradient-image workspace as scratch.  Errors: INVALID_ARG (null pointer, n_new >
 * 2^24, n_old + n_new > capacity, settings out of range, n_pixels * 4096 * n_new >= 9e18), STATE
 * (no views), CUDA. */
SPLAT_API int splat_densify(splat_ctx *ctx, const float *target_depth, const float *depth,
                            const float *alpha, const splat_densify_config *cfg, int64_t n_new,
                            float *pos_logit, float *quat, float *log_scale, int64_t n_old,
                            int64_t capacity, void *stream);

/* Photometric registration residual of a rendered view against a query range image of the same
 * sensor model, with its Gauss-Newton normal equations in the pose (Sec. 3.3.3, Eq. L_photo; the
 * pose update T <- T exp(delta) of that section).  For pixel u of view `view` with
 * O(u) >= o_min: d = D / O, p = d v(u) (render frame), p' = T p (query frame),
 * u' = phi(p') with continuous column c' = (pi - atan2(y', x')) / dgamma - 1/2 and row
 * r' = (elev_max - atan2(z', |x'y'|)) / dtheta; query_depth is sampled bilinearly at u'
 * (columns wrap; the four pixels must exist and be > 0); r = |p'| - Dq(u') (at T = I the
 * printed D(u) - Dq(u) with D read as the range d); J = dr/dxi for T exp(xi^), xi = (rho,
 * omega) in the render frame; Huber IRLS weight w = min(1, huber_delta / |r|).
 * depth, alpha, query_depth: device, the view's rows x cols pixels (for the packed images, the
 * pointer plus the view's first pixel).  T_qm: device float[12], row-major 3 x 4 [R | t]
 * (device-resident so a capturable Gauss-Newton loop can update it).  normal_eqs: device
 * double[29], written: H = sum w J J^T upper triangle row-major (21), g = sum w J r (6), the
 * Huber cost sum, the number of pixels used.  per_pixel (nullable): device float[8][P] planar,
 * r, w, J (zeros where a pixel is not used).  Stream-ordered, no allocation.
 * Errors: INVALID_ARG (null pointer, view out of range, o_min or huber_delta <= 0), STATE (no
 * views), CUDA. */
SPLAT_API int splat_photometric(splat_ctx *ctx, int32_t view, const float *depth,
                                const float *alpha, const float *query_depth, const float *T_qm,
                                float o_min, float huber_delta, double *normal_eqs,
                                float *per_pixel, void *stream);

/* ---- loss and optimiser ------------------------------------------------------------------- */

/* Per-pixel loss over n_pixels packed pixels (depth/alpha/target_depth [P], normal and
 * target_normal [3][P] planar with plane stride n_pixels): valid pixels are those with
 * target_depth > 0 (M_v); L = sum Dt^rho_exp |D - Dt| + lambda_n (1 - N . Nt) + lambda_o (-log
 * max(O, o_eps)).  Writes dL_ddepth, dL_dnormal (3 x P), dL_dalpha (0 outside M_v), and ADDS L to
 * *loss_out (device double; caller zeroes it).  cfg->normal_mode must be SPLAT_NORMALS_TARGET
 * (the range-map mode needs the views: splat_view_loss).  Errors: INVALID_ARG, CUDA. */
SPLAT_API int splat_loss(const float *depth, const float *normal, const float *alpha,
                         const float *target_depth, const float *target_normal,
                         int64_t n_pixels, const splat_loss_config *cfg, float *dL_ddepth,
                         float *dL_dnormal, float *dL_dalpha, double *loss_out, void *stream);

/* The loss of splat_loss over the packed images of the context's registered views (P =
 * ctx's pixel count), with either normal mode of splat_loss_config; every registered view counts
 * (keyframe sampling applies inside splat_refine_step only).  target_normal may be NULL when
 * cfg->normal_mode = SPLAT_NORMALS_RANGE_MAP.  ADDS L to *loss_out.  Stream-ordered.
 * Errors: INVALID_ARG (null pointer, unknown mode), STATE (no views), CUDA. */
SPLAT_API int splat_view_loss(splat_ctx *ctx, const float *depth, const float *normal,
                              const float *alpha, const float *target_depth,
                              const float *target_normal, const splat_loss_config *cfg,
                              float *dL_ddepth, float *dL_dnormal, float *dL_dalpha,
                              double *loss_out, void *stream);

/* One bias-corrected Adam step of n primitives in place: params (pos_logit, quat, log_scale),
 * their gradients (same layout), first and second moments m_*, v_* (same layouts, caller-owned,
 * zero before the first step) and a device int32 step counter that the call increments
 * (the update uses t = *step + 1).  Errors: INVALID_ARG, CUDA. */
SPLAT_API int splat_adam_step(float *pos_logit, float *quat, float *log_scale,
                              const float *g_pos_logit, const float *g_quat,
                              const float *g_log_scale, float *m_pos_logit, float *m_quat,
                              float *m_log_scale, float *v_pos_logit, float *v_quat,
                              float *v_log_scale, int32_t *step, int64_t n,
                              const splat_adam_config *cfg, void *stream);

/* One whole refinement iteration over the registered views, fused:
 * render -> loss against the packed targets -> backward -> Adam, with the chain rule to the
 * parameters fused into the Adam pass (no parameter-gradient buffers).  params are updated in
 * place; m_* / v_* / step as in splat_adam_step; *loss_out receives (is overwritten with) the
 * loss of this iteration.  Capturable in a CUDA graph (no host sync, no allocation).
 * Errors: INVALID_ARG, STATE, CUDA. */
SPLAT_API int splat_refine_step(splat_ctx *ctx, float *pos_logit, float *quat, float *log_scale,
                                int64_t n, const float *target_depth, const float *target_normal,
                                const splat_loss_config *loss_cfg,
                                const splat_adam_config *adam_cfg, float *m_pos_logit,
                                float *m_quat, float *m_log_scale, float *v_pos_logit,
                                float *v_quat, float *v_log_scale, int32_t *step,
                                double *loss_out, void *stream);

/* ---- rendering without allocation -------------------------------------------------------- */

/* The paper has no counterpart to this entry point: it exists for callers that cannot allocate
 * device memory (for instance a process whose device memory is owned by another allocator, or
 * code that must not call cudaMalloc once it is running).  It renders one view like
 * splat_render, with no context: every workspace buffer lives in one array of the library
 * (about 9 MB), and the call allocates nothing -- no cudaMalloc, cudaFree or host heap.
 * The array and the kernels' code take device memory when CUDA loads the library's code on a
 * device, and keep it until the process exits.  CUDA loads that code when it is first used on
 * the device (lazy module loading is CUDA's default), so the FIRST call on each device is a
 * set-up call: it loads the code it uses and looks up the array's device address, with that
 * device current.  Make that first call before handing the device's memory to another
 * allocator, and outside any stream capture; every later call allocates nothing.
 * Limits: g->n <= 16384 primitives, rows <= 256, rows * cols <= 65536 pixels, at most 4096
 * tiles and 262144 (tile, primitive) pairs.  cfg = NULL uses splat_default_config.
 * Outputs: depth[P], normal[3][P], alpha[P] (P = rows * cols), as splat_render.
 * The call waits for its stream before returning.  Errors: INVALID_ARG (null pointer or a size
 * beyond the limits, bad pose or intrinsics), UNSUPPORTED (tile shape), CAPACITY (more pairs
 * than the limit: outputs invalid), NONFINITE (a primitive had a non-finite value: it was
 * skipped), CUDA.  All calls share the one array, which keeps the previous call's contents:
 * calls that overlap on the GPU, or come from several host threads at once, race. */
SPLAT_API int splat_render_noalloc(const splat_gaussians *g, const double T_world_sensor[16],
                                   const splat_lidar_intrinsics *intr,
                                   const splat_render_config *cfg, float *depth, float *normal,
                                   float *alpha, void *stream);

/* ---- status, statistics, inspection ------------------------------------------------------- */

/* Synchronise the device and read (then clear) the status word. */
SPLAT_API int splat_get_status(splat_ctx *ctx, uint32_t *flags);

/* Synchronise the device and read the counters of the last render / backward. */
SPLAT_API int splat_get_stats(splat_ctx *ctx, splat_stats *out);

/* Profiling: when enabled, the next render / backward calls record CUDA events immediately
 * before and after their compositing kernel (forward) and adjoint kernel (backward) on the call's
 * stream; splat_kernel_times then returns those two kernels' durations in milliseconds (waiting
 * for the events), or -1 for a kernel not recorded since profiling was enabled.  Calls made
 * while the stream is being captured into a graph record nothing.  Errors: INVALID_ARG, CUDA. */
SPLAT_API int splat_set_profiling(splat_ctx *ctx, int enable);
SPLAT_API int splat_kernel_times(splat_ctx *ctx, float *fwd_ms, float *bwd_ms);
/* With profiling enabled: the durations (ms, waiting for the events) of the stages of the last
 * profiled render and refinement step, ms[7] = projection, range sort, emission (count, scan,
 * emit), tile sort, tile ranges and work order, loss, fused Adam; -1 for a stage not recorded
 * since profiling was enabled (the last two come from splat_refine_step only).
 * Errors: INVALID_ARG, CUDA. */
SPLAT_API int splat_stage_times(splat_ctx *ctx, float *ms);

/* Copy workspace state of the last render to host memory (synchronising), for tests and
 * profiling.  which = 0: sorted global tile ids (uint32, n_pairs); 1: pair ids of the sorted
 * list (uint32, n_pairs; pair id = view * n + primitive); 2: per-tile [start, end) (uint32 x 2 x
 * n_tiles); 3: per-(view, primitive) records (16 bytes each: int16 row0, row1, col0, ncols;
 * float32 kappa; uint32 bits 0-29 tile count, bit 30 normal flipped, bit 31 invalid input);
 * 4: per-pixel final transmittance (float32, P); 5: per-pixel contributor bound (int32, P).
 * bytes is the size of dst; returns the number of bytes copied, or -1 on error. */
SPLAT_API int64_t splat_debug_copy(splat_ctx *ctx, int32_t which, void *dst, int64_t bytes);

/* Text of a return code. */
SPLAT_API const char *splat_error_string(int code);

/* Text of the last CUDA error seen by any call (thread-local). */
SPLAT_API const char *splat_last_cuda_error(void);

/* Library version (major * 100 + minor). */
SPLAT_API int splat_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPLATLOAM_H */
