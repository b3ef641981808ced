/*
 * gs2 — B300-native hot path of near-second-order (local Newton) 3D Gaussian
 * Splatting training, arXiv 2501.13975 ("3DGS^2").  C ABI of libgs2.so.
 *
 * Conventions for every call
 *  - Device pointers are CUDA device addresses owned by the caller; the
 *    library never frees them.  Host pointers are marked "host".
 *  - Every call that takes a cudaStream_t is asynchronous on that stream.
 *    Argument and shape errors are reported synchronously as a gs2_status;
 *    faults found on the device (pair-capacity overflow, non-finite input)
 *    are recorded in a device status word read by gs2_check().
 *  - No C++ exception crosses this ABI.  A gs2_ctx is not thread-safe: use
 *    one context per host thread / stream.
 *  - Layouts are planar structure-of-arrays in FP32 ("[3][n]" means three
 *    contiguous rows of n floats).  Images are planar [3][H][W].
 *  - Pixel (m, n) of an image has its centre at pixel coordinates (m, n).
 *
 * The method (section / equation of the paper):
 *  Sec. 3 Eq. 3dgs         front-to-back alpha compositing of depth-sorted,
 *                          projected Gaussians (gs2_project, gs2_raster_fwd)
 *  Sec. 4.2 loss eqs.      per-pixel first and diagonal second derivatives of
 *                          L = L2 + lambda L_SSIM (gs2_loss_derivs)
 *  Eq. local_hessian_gradient  per-Gaussian, per-attribute-group gradient and
 *                          Hessian blocks by the chain rule (gs2_accum_newton_blocks)
 *  Eq. local_newton, Sec. 4.2 solves  damped local Newton steps: position in
 *                          the plane perpendicular to the view ray, scaling in
 *                          the projected-eigenvalue subspace, rotation about the
 *                          view ray, opacity with a log barrier, colour per
 *                          channel (gs2_solve_step, gs2_apply_step)
 *  Sec. 4.1, 4.3 Eq. tildel  camera KNN on the bounding sphere; secondary
 *                          targets (downsampled) added to the primary's blocks
 *                          (gs2_camera_knn, gs2_sweep)
 */
#ifndef GS2_H
#define GS2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *gs2_stream; /* same type as cudaStream_t */
typedef struct gs2_ctx gs2_ctx;

typedef enum {
    GS2_OK = 0,
    GS2_ERR_ARG = 1,         /* null pointer, bad enum, bad config value */
    GS2_ERR_SHAPE = 2,       /* size beyond what the context was created for */
    GS2_ERR_CUDA = 3,        /* a CUDA runtime call failed (see gs2_last_error) */
    GS2_ERR_OOM = 4,         /* scratch allocation failed in gs2_create */
    GS2_ERR_NONFINITE = 5,   /* device status: non-finite value met */
    GS2_ERR_TIMEOUT = 6,     /* device status: a bounded device wait gave up */
    GS2_ERR_UNSUPPORTED = 7, /* e.g. SH degree > 3 */
    GS2_ERR_CAPACITY = 8     /* device status: more tile/Gaussian pairs than max_pairs */
} gs2_status;

/* Attribute groups, solved in this order within a sweep (Sec. 4.2). */
typedef enum { GS2_POS = 0, GS2_ROT = 1, GS2_SCALE = 2, GS2_OPACITY = 3, GS2_COLOR = 4 } gs2_group;

/* Scene: caller-owned device buffers, FP32, planar SoA.
 *   mean    [3][n]   world positions p
 *   quat    [4][n]   unit quaternions (w, x, y, z)
 *   scale   [3][n]   linear axis scales s (> 0)
 *   opacity [n]      sigma in (0, 1)
 *   sh      [3][S][n] SH coefficients per channel, S = (sh_degree + 1)^2 */
typedef struct {
    int32_t n;
    int32_t sh_degree;
    float *mean;
    float *quat;
    float *scale;
    float *opacity;
    float *sh;
} gs2_scene;

/* Pinhole camera looking along +z of its frame (x right, y down).
 * viewmat: host, row-major 3x4 [R | t], world -> camera.
 * pi = (fx tx/tz + cx, fy ty/tz + cy) in pixels for t = R p + t.
 * clip_x, clip_y: limits of tx/tz, ty/tz inside the projection Jacobian of the
 *   EWA covariance (the standard 3DGS frustum clamp); 0 selects
 *   1.3 * (width/2) / fx and 1.3 * (height/2) / fy of this camera. */
typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float viewmat[12];
    float clip_x, clip_y;
} gs2_camera;

/* Configuration.  Every constant the paper leaves unstated is a field; the
 * defaults (gs2_config_default) are this library's readings of them. */
typedef struct {
    float lambda_ssim;      /* weight of the SSIM loss (0.2) */
    float alpha_min;        /* skip terms with alpha < alpha_min (1/255) */
    float alpha_max;        /* alpha = min(sigma G, alpha_max) (0.99) */
    float t_min;            /* stop before T falls below t_min (1e-4) */
    float lowpass;          /* screen-space low-pass added to Sigma2D (0.3) */
    float near_z;           /* cull centres with camera depth < near_z (0.2) */
    float barrier_alpha;    /* opacity log-barrier weight (1e-6) */
    float frac_to_boundary; /* opacity fraction-to-boundary tau (0.99) */
    float damping_mu0;      /* first damping factor mu0 (1.0) */
    int32_t damping_tries;  /* extra x10 damping attempts (6) */
    float scale_min;        /* floor of any scale (1e-7) */
    float scale_trust;      /* scale update bounded to [s/k, k s] (1.05) */
    float trust_pos;        /* |dp| <= trust_pos * max(s) (0.05) */
    float trust_rot;        /* |theta| <= trust_rot (0.05) */
    float trust_color;      /* per-channel SH step norm <= trust_color (0.05) */
    float ssim_c1, ssim_c2; /* 0.01^2, 0.03^2 */
    float ssim_sigma;       /* Gaussian window sigma (1.5) */
    int32_t ssim_radius;    /* window radius (5: 11x11); only 5 is supported */
    int32_t knn_k;          /* secondary targets per primary (3) */
    int32_t downsample;     /* secondary-target downsampling factor (2) */
    int32_t precision;      /* 0: FP32 path; 1: mixed (FP64 solve of ill-conditioned blocks) */
    int32_t gauss_newton;   /* 0: full local Newton blocks (Eq. local_hessian_gradient); 1: drop the
                               e d2c/dy2 terms, keeping sum h dc/dy dc/dy^T (local Gauss-Newton, the
                               cheaper variant Sec. 6 proposes; positive semidefinite where h >= 0) */
    int32_t group_order[5]; /* the groups of a sweep in the order run: a permutation of gs2_group
                               (0 1 2 3 4 = position, rotation, scaling, opacity, colour: Sec. 4.2;
                               Sec. 5 compares orders) */
    int32_t group_jacobi;   /* 0: the groups in series, every view re-rendered after each group's
                               step (Sec. 4.2); 1: every view rendered once per sweep, all groups'
                               blocks accumulated from it, solved at that state and applied together
                               (Jacobi over groups, position applied last).  Setting it allocates
                               the per-group blocks and steps in gs2_create / gs2_set_config; the
                               step-scale network and the logged sweep need the series form. */
    float gd_lr[5];         /* per group (gs2_group index): 0 = the damped Newton step (the paper);
                               > 0 = the first-order baseline, step -gd_lr g of the group's gradient
                               (opacity with the barrier's), inside the same trust radii and bounds
                               (position as a full 3D step) */
    int32_t deterministic;  /* 0: block sums with float atomics (order of additions not fixed);
                               1: identical bytes on every run: each (tile, Gaussian) entry of the
                               tile lists gets its own partial sum (the tile's four warp sums added
                               in warp order, no atomics), each Gaussian's entries are then summed in
                               emission order (compensated FP32, or FP64 with precision = 1), and the
                               views of a sweep run one after another.  Setting it allocates
                               max_pairs x 41 floats of partials and three max_pairs index arrays in
                               gs2_create / gs2_set_config (7.9 GB at 48M pairs). */
    float learned_trust;    /* with a step-scale network installed: the learned step alpha d may reach
                               learned_trust times the trust radii (scale bounds [s / k^lt, k^lt s]),
                               so that it can lengthen a step the plain radius clipped (1: the plain
                               radii; 2 measured worse on the object workload) */
} gs2_config;

void gs2_config_default(gs2_config *cfg);

/* Context: owns only scratch (sorting buffers, tile ranges, per-view
 * image-space accumulators, per-pixel loss derivatives, sweep buffers).
 * max_pairs: capacity of the (tile, Gaussian) pair list per view (0 picks
 * 16 * max_gaussians).  Limits: max_width * max_height <= 2^28 pixels and
 * each side at most 1,048,560 pixels (65,535 tiles of 16: tile coordinates
 * are 16-bit), else GS2_ERR_SHAPE, checked before any device call.  Returns
 * GS2_ERR_OOM if scratch cannot be allocated.
 * Creates scratch on the current CUDA device. */
gs2_status gs2_create(gs2_ctx **out, const gs2_config *cfg, int64_t max_gaussians, int32_t max_width,
                      int32_t max_height, int32_t max_sh_degree, int64_t max_pairs);
gs2_status gs2_destroy(gs2_ctx *ctx);
const char *gs2_last_error(const gs2_ctx *ctx);
gs2_status gs2_set_config(gs2_ctx *ctx, const gs2_config *cfg);

/* Synchronises the stream, returns and clears the device status word
 * (GS2_OK, GS2_ERR_CAPACITY, GS2_ERR_NONFINITE, GS2_ERR_TIMEOUT). */
gs2_status gs2_check(gs2_ctx *ctx, gs2_stream stream);

/* Sizes of caller-owned buffers, in bytes. */
size_t gs2_proj_bytes(int64_t n);
size_t gs2_raster_state_bytes(int32_t width, int32_t height);
/* Blocks of one group for n Gaussians; colour keeps one factored slot per view
 * (n_views = 1 + knn_k in a sweep). */
size_t gs2_blocks_bytes(gs2_group group, int64_t n, int32_t sh_degree, int32_t n_views);
size_t gs2_step_bytes(gs2_group group, int64_t n, int32_t sh_degree);

/* Projection of every Gaussian into one view (Sec. 3; App. A.1-A.3):
 * centre pi, EWA covariance Sigma2D = J Wr R S S^T R^T Wr^T J^T + lowpass I
 * with J the perspective Jacobian, its inverse (conic), view-dependent SH
 * colour c~ (App. A.2), depth key and screen-tile rectangle of the support
 * { sigma G >= alpha_min }.  proj: device, gs2_proj_bytes(n) bytes, opaque.
 * A Gaussian with a non-finite parameter is left off screen and the device
 * status gets GS2_ERR_NONFINITE's bit (read by gs2_check). */
gs2_status gs2_project(gs2_ctx *ctx, const gs2_scene *scene, const gs2_camera *cam, void *proj,
                       gs2_stream stream);

/* Tile binning, per-tile depth sort (key = FP32 camera depth, ties by index)
 * and front-to-back compositing, Eq. 3dgs:
 *   c = sum_k alpha_k c~_k prod_{j<k} (1 - alpha_j),  alpha = min(sigma G, alpha_max),
 * terms with alpha < alpha_min skipped, stop before T < t_min, black background.
 * image: device [3][H][W] out.  raster_state: device, gs2_raster_state_bytes,
 * out (final transmittance and per-pixel list length).  The sorted tile lists
 * stay in ctx until the next gs2_raster_fwd on this ctx. */
gs2_status gs2_raster_fwd(gs2_ctx *ctx, const gs2_scene *scene, const gs2_camera *cam, const void *proj,
                          float *image, void *raster_state, gs2_stream stream);

/* Per-pixel loss derivatives (Sec. 4.2 loss equations):
 *   e = dL/dc and h = d2L/dc_q^2 (pixel-diagonal) of L = L2 + lambda L_S,
 *   L2 = 1/(3|I|) sum 1/2 (c - c^t)^2, L_S = 1/(3|I|) sum (1 - SSIM), SSIM per
 *   channel with an 11x11 Gaussian window, zero-padded.
 * image, target: device [3][H][W]; e, h: device [3][H][W] out;
 * loss_out: device double[2] (L2, L_S) accumulated (+=), may be NULL.
 * A non-finite pixel of image or target counts as 0 and sets the status bit
 * of GS2_ERR_NONFINITE. */
gs2_status gs2_loss_derivs(gs2_ctx *ctx, const float *image, const float *target, int32_t width,
                           int32_t height, float *e, float *h, double *loss_out, gs2_stream stream);

/* Gradient and Hessian blocks of one group from one view (Eq.
 * local_hessian_gradient, full Newton: g = sum e dc/dy,
 * H = sum (dc/dy)^T diag(h) dc/dy + e . d2c/dy2), added into blocks.
 * Must follow gs2_raster_fwd of the same view on this ctx (uses its tile
 * lists).  primary: the primary view, which fixes the rotation axis.
 * image: device [3][H][W], this view's gs2_raster_fwd output; target: device
 * [3][H][W] of this view; the per-pixel derivatives are formed internally
 * (as gs2_loss_derivs).  loss_out as gs2_loss_derivs.
 * blocks (device, gs2_blocks_bytes), layout:
 *   POS, SCALE: g [3][n], H [6][n] (upper triangle 00 01 02 11 12 22)
 *   ROT, OPACITY: g [1][n], H [1][n]
 *   COLOR: slot v (= view_slot) of n_views: [a_ch (3), s_ch (3), b (S)][n] with
 *          a_ch = sum_p w e_ch, s_ch = sum_p w^2 h_ch, b = B Phi(r_v); the
 *          channel block is H_ch = sum_v s_ch b b^T, g_ch = sum_v a_ch b.
 *          The dense S x S block is never formed: gs2_solve_step solves each
 *          channel in the range of the (at most 4) view bases b_v, an r x r
 *          system, so the SH J^T J contraction has no dense product to put on
 *          the tensor cores (BF16 or otherwise).
 *          The slot is overwritten, other groups accumulate (+=). */
gs2_status gs2_accum_newton_blocks(gs2_ctx *ctx, gs2_group group, const gs2_scene *scene,
                                   const gs2_camera *view, const gs2_camera *primary, const void *proj,
                                   const void *raster_state, const float *image, const float *target,
                                   int32_t view_slot, void *blocks, double *loss_out, gs2_stream stream);

/* Damped local Newton step per Gaussian (Eq. local_newton), H + mu m I with
 * m = mean |diag H| and mu = mu0 10^i until Cholesky succeeds; reduced
 * bases from the primary view: position in span(U), U perpendicular to the
 * view ray; scaling in the row space of d lambda / d s (projected
 * eigenvalues); rotation angle about the view ray; opacity with barrier and
 * fraction-to-boundary; colour per channel.
 * step: device, gs2_step_bytes.  n_failed: device int, incremented by the
 * number of blocks whose damping ladder failed (their step is 0). */
gs2_status gs2_solve_step(gs2_ctx *ctx, gs2_group group, const void *blocks, int32_t n_views,
                          const gs2_scene *scene, const gs2_camera *primary, void *step, int32_t *n_failed,
                          gs2_stream stream);

/* Update in place (Sec. 4.2): p += dp; q <- dq(theta) (x) q with dq the
 * rotation by theta about the primary view ray, renormalised;
 * s <- max(s + ds, scale_min); sigma += dsigma; c += dc. */
gs2_status gs2_apply_step(gs2_ctx *ctx, gs2_group group, const void *step, gs2_scene *scene,
                          const gs2_camera *primary, gs2_stream stream);

/* f x f box downsampling of a [3][H][W] image (secondary targets, Sec. 4.3)
 * to [3][H/f][W/f]; the matching camera (host) keeps pixel centres aligned. */
gs2_status gs2_downsample(gs2_ctx *ctx, const float *in, int32_t width, int32_t height, int32_t f, float *out,
                          gs2_stream stream);
void gs2_camera_downsample(const gs2_camera *in, int32_t f, gs2_camera *out);

/* Data preparation (Sec. 4.1): bounding sphere of the means (centre of their
 * bounding box, radius = largest distance to a mean): sphere_out device
 * float[4].  Camera KNN (host): centres [ncam][3], sphere [4], out [ncam][k]
 * by great-circle distance of the radially projected centres, ties by index. */
gs2_status gs2_bounding_sphere(gs2_ctx *ctx, const gs2_scene *scene, float *sphere_out, gs2_stream stream);
gs2_status gs2_camera_knn(const float *centres, int32_t ncam, const float *sphere, int32_t k, int32_t *out);

/* One sweep for primary image t (Sec. 4.2 group order, Sec. 4.3 Eq. tildel):
 * for each group in cfg.group_order, render the primary (full resolution) and
 * its k secondaries (downsampled), accumulate, solve, apply.  The views of a
 * group run concurrently on the context's view lanes (tuning.view_lanes).
 * The configuration selects the variants: cfg.gauss_newton (Gauss-Newton
 * blocks), cfg.gd_lr (gradient steps instead of Newton's for the groups with
 * a positive rate), cfg.group_jacobi (every view rendered once, all groups
 * solved at that state and applied together, position last).  Uses only ctx
 * scratch.  cams: host [ncam]; targets: host array of ncam device pointers to
 * full-resolution [3][H][W] images (only the primary's and its secondaries'
 * entries are read); knn: host [ncam][knn_k].
 * losses_out: device double[5][2], (L2, L_S) of the primary view seen by each
 * group, indexed by group (+=; with group_jacobi only the slot of the first
 * group of the order, from the sweep's single render), may be NULL.
 * n_failed: device int (+=), may be NULL. */
gs2_status gs2_sweep(gs2_ctx *ctx, gs2_scene *scene, const gs2_camera *cams, int32_t ncam,
                     const float *const *targets, const int32_t *knn, int32_t t, double *losses_out,
                     int32_t *n_failed, gs2_stream stream);

/* Learned step scale (an extension; the paper's local Newton step has step
 * size 1, Sec. 4.2).  A 8-64-64-1 MLP (ReLU; BF16 weights, FP32 accumulation)
 * maps 8 features of a Gaussian's plain damped step d to alpha = 2 sigmoid(y)
 * in (0, 2); the step becomes alpha d, limited by the same trust radii and
 * bounds as d.  The plain step stays wherever the features are unusable
 * (|d| = 0, g . d >= 0, a non-finite value) or alpha is not finite.
 *
 * Records: float [GS2_REC_ROWS][n] per group and sweep: rows 0-7 the
 * features, row 8 phi0, row 9 the label alpha* in [0, 2] or -1 for an
 * unusable record, row 10 phi1.  The label looks along d at a loss L_lab: phi0 = grad
 * L_lab . d before the step, phi1 = grad L_lab . d after all Gaussians of the
 * group stepped; alpha* = 0 if phi0 >= 0 (d does not descend L_lab: a
 * rejected step), else the minimum of the quadratic line model
 * phi0 / (phi0 - phi1) (2 where that model is not convex), clipped to
 * [0, 2].  gs2_step_records/gs2_step_labels use the loss of the blocks passed
 * (phi0 = g . d); gs2_sweep_logged uses the loss summed over every training
 * view at full resolution, whose increase is the overshoot of Sec. 4.3.
 * Features (g, H the group's block, g_p the primary view's own gradient):
 *   f0 log10 clamp(d^T H d / (-g.d), 1e-6, 1e6)   f1 cos(-g, d)
 *   f2 log10 max(|d|/u, 1e-12), u = max(s) for position and scaling, else 1
 *   f3 sigma   f4 clamp(g_p.d / g.d, -4, 4) (0 if g.d >= 0)
 *   f5 1 if a trust radius or bound is within 1e-3 of limiting d, else 0
 *   f6 log10 clamp(|g| / (mean|diag H| |d|), 1e-6, 1e6)   f7 group / 4
 * g_p: gs2_accum_newton_blocks keeps the gradient rows of blocks as they are
 * right after a view_slot 0 accumulation in the context (colour: slot 0 of
 * its blocks); accumulate the primary view in slot 0, first.
 * Parameters (GS2_MLP_NPARAM words): W1 [64][8], b1 [64], W2 [64][64],
 * b2 [64], W3 [64], b3. */
#define GS2_MLP_NFEAT 8
#define GS2_MLP_HIDDEN 64
#define GS2_MLP_NPARAM 4801
#define GS2_MLP_GRID 148
#define GS2_REC_ROWS 11

/* Install (device, GS2_MLP_NPARAM BF16 words, read at every solve; the caller
 * keeps it alive) or remove (NULL) the step-scale network: gs2_solve_step and
 * gs2_sweep then scale each step after the plain solve.  With a network
 * installed (this one or the damping network) a sweep's view lanes add their
 * epilogues into blocks of their own, summed after the join, so that the
 * primary view's gradient (feature f4) is taken before any secondary adds to
 * the blocks; the first install allocates those blocks (one view's blocks
 * per lane), so it does not belong in a stream capture. */
gs2_status gs2_set_step_model(gs2_ctx *ctx, const uint16_t *w_bf16);

/* Records of the plain step: features and phi0 of step (from blocks, as
 * passed to gs2_solve_step), label row set to 0 (pending) or -1 (unusable).
 * records: device float [GS2_REC_ROWS][scene->n] out. */
gs2_status gs2_step_records(gs2_ctx *ctx, gs2_group group, const void *blocks, int32_t n_views,
                            const gs2_scene *scene, const void *step, float *records, gs2_stream stream);
/* Labels: blocks_after are the group's blocks accumulated over the same views
 * after the step was applied; fills row 9 of the pending records. */
gs2_status gs2_step_labels(gs2_ctx *ctx, gs2_group group, const void *blocks_after, int32_t n_views,
                           const gs2_scene *scene, const void *step, float *records, gs2_stream stream);
/* gs2_sweep of the plain method (installed networks are not used) that
 * also logs every group's records, labelled by the loss over all ncam views
 * at full resolution (every view is accumulated before and after the step;
 * all cameras must fit the context).  records: device float
 * [5][GS2_REC_ROWS][n] out.  records_damping (may be NULL): device float
 * [5][GS2_REC_ROWS][n] out, the damping network's records (see
 * gs2_set_damping_model); the first call that passes it allocates the
 * labels' scratch (so it is not for stream capture).  The scene ends as
 * after gs2_sweep. */
gs2_status gs2_sweep_logged(gs2_ctx *ctx, gs2_scene *scene, const gs2_camera *cams, int32_t ncam,
                            const float *const *targets, const int32_t *knn, int32_t t, float *records,
                            float *records_damping, double *losses_out, int32_t *n_failed, gs2_stream stream);

/* Learned damping (an extension; the paper is silent on damping, Sec. 4.2).
 * A second network of the same shape, layout and features maps a Gaussian's
 * plain damped step to a multiplier rho = 10^(1.5 alpha) in (1, 1e3) of the
 * damping mu0 (alpha = 2 sigmoid(y): the damping can only grow, where the
 * measured gain of the best candidates lies); for the position, scaling and
 * colour groups, whose damping turns the step and not only shortens it,
 * gs2_solve_step and gs2_sweep then solve again with mu0 rho (the rotation
 * and opacity blocks are 1 x 1: there damping and step scale coincide).  The
 * plain solve's rho stays 1 where the features are unusable or alpha is not
 * finite.  An installed step-scale network then scales the re-solved step.
 * Its records (gs2_sweep_logged) carry the step records' features and, in
 * row 9, the label 2 log10(rho*) / 3, rho* the multiplier among
 * 10^0, 10^0.5, ..., 10^3 whose step (the same damped solve, trust radii and bounds)
 * has the smallest quadratic model of the loss over every training view,
 * Q(d) = g_all . d + 1/2 d^T H_all d (the group's blocks accumulated over
 * every view at full resolution before the step; smallest rho on ties); -1
 * where the step record is unusable, no candidate has Q < 0, or the group's
 * damping is not learned.  Rows 8 and 10 hold phi0 = -w a* and phi1 = phi0 + w
 * (a* the label, w = the largest minus the smallest finite Q of the
 * candidates; 0 without a label), so that gs2_mlp_grad's line objective
 * becomes sum s_c w (a^2 / 2 - a* a): the label loss weighted by how much the
 * record's choice of damping changes Q.  It is trained with gs2_mlp_grad
 * (labels or line) and gs2_mlp_adam like the step-scale network.
 * Install (device, GS2_MLP_NPARAM BF16 words, read at every solve; the caller
 * keeps it alive) or remove (NULL); installing allocates as
 * gs2_set_step_model does. */
gs2_status gs2_set_damping_model(gs2_ctx *ctx, const uint16_t *w_bf16);

/* Network training and evaluation on record buffers made of chunks
 * [GS2_REC_ROWS][chunk_n] (row j of record i at
 * records[(i / chunk_n) GS2_REC_ROWS chunk_n + j chunk_n + i % chunk_n]);
 * record r of a batch is idx[r] (device int64, NULL: r).
 * gs2_mlp_forward: out[r] = alpha(features of record r), device float [nrec].
 * gs2_mlp_grad: over the usable records (label >= 0) the loss
 *   1/2 sum (alpha - alpha*)^2 (chunk_scale NULL), or, with chunk_scale
 *   (device float, one per chunk), the line model's predicted change of the
 *   label loss sum s_c (phi0 alpha + 1/2 (phi1 - phi0) alpha^2);
 *   partial: device float [GS2_MLP_GRID][GS2_MLP_NPARAM] out,
 *   per-CTA gradient sums w.r.t. the BF16 weights' values; stats: device
 *   double [GS2_MLP_GRID][2] out, per-CTA (loss, usable count).
 * gs2_mlp_adam: one Adam step of the FP32 master weights with the mean
 *   gradient (sum of partial rows / usable count; no change if the count is
 *   0), then w_bf16 = round-to-nearest-even BF16 of master.  m, v: device
 *   float [GS2_MLP_NPARAM] moments; step >= 1 is the Adam step number. */
gs2_status gs2_mlp_forward(const uint16_t *w_bf16, const float *records, int64_t chunk_n, const int64_t *idx,
                           int64_t nrec, float *out, gs2_stream stream);
gs2_status gs2_mlp_grad(const uint16_t *w_bf16, const float *records, int64_t chunk_n, const int64_t *idx,
                        int64_t nrec, const float *chunk_scale, float *partial, double *stats, gs2_stream stream);
/* Per-chunk scale of the line-model loss: out[c] = 1 / sum over the usable
 * records of chunk c of |phi0| (0 if none); out: device float [n_chunks]. */
gs2_status gs2_records_chunk_scale(const float *records, int64_t chunk_n, int64_t n_chunks, float *out,
                                   gs2_stream stream);
gs2_status gs2_mlp_adam(float *master, uint16_t *w_bf16, const float *partial, const double *stats, float *m,
                        float *v, int32_t step, float lr, float beta1, float beta2, float eps, gs2_stream stream);

/* Kernel tuning of a context (no effect on results beyond the order of
 * floating-point additions: the sort is stable and exact for every setting).
 *   sort_blocks: CTAs of every radix-sort pass (1..1024; default 592)
 *   sort_rows:   keys per thread per scatter round (2, 4, 8 or 16; default 4)
 *   view_lanes:  1 (default): a sweep runs the views of each group
 *                concurrently on streams of the context (one per secondary);
 *                0: one after another on the caller's stream
 *   accum_px:    pixels per thread of the position- and colour-group
 *                accumulations: 4 (default with 16x16 tiles; a warp per 8x16
 *                column of the tile, one warp reduction of the payload per
 *                128 pixels, two warps per tile) or 2 (a warp per 8x8 block,
 *                one reduction per 64 pixels; the only choice with 8x8 tiles
 *                and in deterministic mode).  The rotation, scaling and
 *                opacity groups always take 2.  Same sums, added in another
 *                order.
 *   accum_split: 0 (default): the accumulation runs one CTA per tile over the
 *                tile's whole back-to-front walk.  A multiple of the tile's
 *                pixel count (256 with 16x16 tiles, at most 2^20): every
 *                walk is cut into work items of that many list entries,
 *                which a persistent grid takes longest tiles first, so that a
 *                few long walks no longer bound the launch (dense scenes at
 *                low resolution).  gs2_raster_fwd then also writes, at every
 *                multiple of accum_split entries of a tile's list, each
 *                pixel's T there and the colour its entries from there on add
 *                (checkpoints in ctx); an item starts a pixel whose last
 *                contributor lies behind the item's end from there.  Same
 *                sums, added in another order, with T and the colour behind
 *                rounded differently.  Not used in deterministic mode.
 *                gs2_set_tuning allocates the checkpoints (16 * 256 bytes per
 *                accum_split pairs of max_pairs, plus the item list) for ctx
 *                and its view lanes: it synchronises the device and must not
 *                run under stream capture; GS2_ERR_OOM if they do not fit.
 * gs2_autotune times `reps` sweeps with primary t for every candidate
 * (sort_blocks 296, 592, 888 x sort_rows 2, 4, 8, 16 at the current accum_px
 * and accum_split, then the other accum_px at the best of those, then
 * accum_split 0, 1 and 4 times the tile's pixel count at the best of those;
 * view_lanes kept) on a scratch copy of the scene (the caller's scene
 * is not changed), keeps the fastest in ctx and returns it and its ms per
 * sweep (host outputs, may be NULL).  It allocates the copy and the split
 * checkpoints, synchronises the stream and must not run under stream
 * capture. */
typedef struct {
    int32_t sort_blocks;
    int32_t sort_rows;
    int32_t view_lanes;
    int32_t accum_px;
    int32_t accum_split;
} gs2_tuning;
gs2_status gs2_get_tuning(const gs2_ctx *ctx, gs2_tuning *out);
gs2_status gs2_set_tuning(gs2_ctx *ctx, const gs2_tuning *tuning);
gs2_status gs2_autotune(gs2_ctx *ctx, const gs2_scene *scene, const gs2_camera *cams, int32_t ncam,
                        const float *const *targets, const int32_t *knn, int32_t t, int32_t reps, gs2_tuning *best,
                        float *best_ms, gs2_stream stream);

/* Batched sweeps over independent scenes (an extension: the paper trains one
 * scene at a time).  A batch owns one context and one stream per scene
 * (created with cfg and the scene's maxima).  gs2_batch_sweep runs one
 * gs2_sweep per scene (scene i: scenes[i], cams[i][ncam[i]], targets[i][],
 * knn[i][], primary t[i]; host arrays of n_scenes entries), all forked from
 * `stream` onto the scenes' streams and joined back, so the scenes' kernels
 * share the GPU.  losses_out: device double [n_scenes][10] (+=) or NULL;
 * n_failed: device int [n_scenes] (+=) or NULL.  use_graph = 1 captures the
 * fork/join as one CUDA graph (on a stream of the batch, so `stream` may be
 * the legacy default stream) and launches it on `stream`; the instantiated
 * graph is kept and updated in place on later calls (re-instantiated if the
 * update is refused).  use_graph = 2 keeps one instantiated graph per scene
 * and sweep inputs (a hash of the primary, its views' cameras and target
 * pointers, the scene, output pointers, configuration, step model and
 * tuning; up to 512 per scene): a sweep seen before is replayed without
 * capture, a new one is captured once.  A context's first use must not be under capture: create the
 * batch before capturing anything.  gs2_batch_ctx gives scene i's context
 * (for tuning or checks); gs2_batch_stats the graph instantiation, update
 * and replay counts. */
typedef struct gs2_batch gs2_batch;
typedef struct {
    int64_t max_gaussians;
    int32_t max_width, max_height, max_sh_degree;
    int64_t max_pairs;
} gs2_batch_scene;
gs2_status gs2_batch_create(gs2_batch **out, const gs2_config *cfg, int32_t n_scenes, const gs2_batch_scene *desc);
gs2_status gs2_batch_destroy(gs2_batch *batch);
gs2_ctx *gs2_batch_ctx(gs2_batch *batch, int32_t i);
const char *gs2_batch_last_error(const gs2_batch *batch);
gs2_status gs2_batch_stats(const gs2_batch *batch, int32_t *instantiations, int32_t *updates, int32_t *replays);
gs2_status gs2_batch_sweep(gs2_batch *batch, gs2_scene *scenes, const gs2_camera *const *cams, const int32_t *ncam,
                           const float *const *const *targets, const int32_t *const *knn, const int32_t *t,
                           double *losses_out, int32_t *n_failed, int32_t use_graph, gs2_stream stream);

/* Instrumentation.
 * gs2_launch_count: kernels launched by this library in this process so far.
 * gs2_profile(ctx, 1): from now on record CUDA events around every
 *   accumulation kernel launch and around every binning (depth and tile
 *   sort), compositing and loss-derivative stage (one bounded pool of 2048
 *   event pairs), and count, per group slot of gs2_sweep, the (tile,
 *   Gaussian) pairs, visible Gaussians, binnings and pixels (device-side
 *   counters, no host synchronisation); resets totals.  gs2_profile(ctx, 0)
 *   stops.  Synchronises the device.  Event durations of views that run
 *   concurrently overlap: time with tuning.view_lanes = 0 for per-stage
 *   figures.
 * gs2_profile_read: per group (host arrays [5], stats [5][6]: sorted pairs
 *   (one per tile of each support rectangle), visible Gaussians, binnings,
 *   pixels, accumulation evaluations = (pixel, Gaussian) pairs with alpha >=
 *   alpha_min that the accumulation processed, listed pairs (those whose tile
 *   the support ellipse reaches: the tile lists' total length)) after
 *   synchronising the device.
 * gs2_profile_read_stages: host arrays [3] (binning, compositing, loss
 *   derivatives): summed event milliseconds and the number of timed stages,
 *   after synchronising the device. */
uint64_t gs2_launch_count(void);
gs2_status gs2_profile(gs2_ctx *ctx, int32_t enable);
gs2_status gs2_profile_read(gs2_ctx *ctx, double *accum_ms, int64_t *accum_launches, uint64_t *stats);
gs2_status gs2_profile_read_stages(gs2_ctx *ctx, double *ms_out, int64_t *count_out);

/* Mixed precision (config.precision = 1): the number of blocks (colour: of
 * channels) that gs2_solve_step and the sweeps of this context solved again in
 * FP64 because the FP32 factor's condition estimate (max L_ii / min L_ii)^2
 * exceeded 1e6 or the FP32 damping ladder failed, per group (host out[5]),
 * since creation or the last reset (reset != 0 clears them).  Synchronises the
 * device. */
gs2_status gs2_fp64_resolves(gs2_ctx *ctx, uint64_t *out, int32_t reset);

/* No-allocation render (the paper has no counterpart; this serves callers).
 * Some callers cannot call cudaMalloc: a plugin or callback run by a host
 * application that owns all device memory and does not let its plugins
 * allocate, or a real-time loop that must not pay allocation latency or risk
 * running out of memory halfway through a run.  gs2_render_noalloc does what
 * gs2_project followed by gs2_raster_fwd does for one view, with no gs2_ctx
 * and no allocation: its sorting scratch is one fixed array of
 * GS2_NOALLOC_SCRATCH_BYTES compiled into the library, held on every GPU that
 * loads the library until the process exits.
 *   Limits: at most GS2_NOALLOC_MAX_TILES 16x16 tiles (GS2_ERR_SHAPE beyond)
 *   and GS2_NOALLOC_MAX_PAIRS (tile, Gaussian) pairs; more pairs set
 *   GS2_ERR_CAPACITY's bit (1) in *status_out and the image is then incomplete.
 *   cfg: host, NULL for the defaults; a configuration that gs2_create would
 *   refuse returns GS2_ERR_ARG before any device call.  proj: device,
 *   gs2_proj_bytes(n); image, raster_state: device outputs as for
 *   gs2_raster_fwd; status_out: device uint32, written by every call (0 = OK,
 *   else the status bits of this call only).  status_out may be NULL, but then
 *   a pair overflow cannot be detected at all (there is no context for
 *   gs2_check): an incomplete image still returns GS2_OK.  Pass a status word
 *   unless the scene is known to stay within the limits.
 *   The first call on a device looks up the array's device address with that
 *   device current; make it before any stream capture.  All calls share the
 *   array and leave their contents in it: calls that overlap on the GPU race
 *   and must be serialised by the caller. */
#define GS2_NOALLOC_MAX_PAIRS 524288
#define GS2_NOALLOC_MAX_TILES 4096
#define GS2_NOALLOC_SCRATCH_BYTES 9037312ull
gs2_status gs2_render_noalloc(const gs2_config *cfg, const gs2_scene *scene, const gs2_camera *cam, void *proj,
                              float *image, void *raster_state, uint32_t *status_out, gs2_stream stream);

/* Introspection for tests: copies the current tile ranges (device uint32
 * [ntiles][2]) and sorted Gaussian ids (device uint32, up to capacity) and
 * returns the number of listed pairs (host; the tile lists' total length)
 * after synchronising the stream. */
gs2_status gs2_debug_tiles(gs2_ctx *ctx, uint32_t *ranges_out, uint32_t *ids_out, int64_t capacity,
                           int64_t *n_pairs_out, gs2_stream stream);
/* Test of the device-side bounded wait (fault-free failure detection): the
 * look-back wait of the tiles-touched scan (one warp; Sec. 3 binning) is run
 * from chunk `chunk` (1..255) over look-back states that no chunk publishes
 * (the context's scan state, cleared on `stream` first).  After `limit` polls
 * (1..2^20; the scan itself allows 2^20, about a second) it gives up and sets
 * the status bit that gs2_check reports as GS2_ERR_TIMEOUT; the context stays
 * usable.  Asynchronous on `stream`. */
gs2_status gs2_debug_lookback_timeout(gs2_ctx *ctx, int32_t chunk, uint32_t limit, gs2_stream stream);
/* Depth keys (FP32 bit patterns) written by the last gs2_project into proj. */
gs2_status gs2_debug_keys(const void *proj, int64_t n, uint32_t *keys_out, gs2_stream stream);
/* Unpacks proj into planar FP32 [GS2_DEBUG_PROJ_ROWS][n]: pix_x pix_y conic_xx
 * conic_xy conic_yy sigma col0 col1 col2 depth tiles_touched(as float) l lmax
 * k2 ry rect.x rect.y 0, where l, lmax are the thresholds of the quadratic
 * form (composited iff q <= l, clamped iff q < lmax), k2 = det Sigma2D /
 * Sigma_yy^2, ry the padded half height of the support box and rect.x, rect.y
 * the tile rectangle's two words (tx0 | ty0 << 16, tx1 | ty1 << 16, exclusive
 * ends) stored as their bit patterns. */
#define GS2_DEBUG_PROJ_ROWS 18
gs2_status gs2_debug_proj(const void *proj, int64_t n, float *out, gs2_stream stream);

#ifdef __cplusplus
}
#endif
#endif
