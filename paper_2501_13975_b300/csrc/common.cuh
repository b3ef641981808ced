// Internal declarations shared by the gs2 CUDA translation units.
// Not part of the public ABI (include/gs2.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <string>

#include "../../include/gs2.h"
#include "decide.cuh"

// screen tile edge in pixels: 16, or 8 in a build with -DGS2_TILE=8 (a
// measurement variant; the tile size is fixed per build)
#ifndef GS2_TILE
#define GS2_TILE 16
#endif
#if GS2_TILE != 8 && GS2_TILE != 16
#error "GS2_TILE must be 8 or 16"
#endif
#define GS2_SORT_BLOCKS_MAX 1024     // the per-digit scan runs one 1024-thread CTA per digit
#define GS2_SPLIT_MAX (1 << 20)      // largest work item of the split accumulation (list entries)
// profiling pool (event pairs) and the stage tags beside the accumulation groups
#define GS2_PROF_POOL 2048
#define GS2_PROF_BIN 5
#define GS2_PROF_RASTER 6
#define GS2_PROF_LOSS 7
#define GS2_MAX_LANES 16             // concurrent views per group in a sweep (secondaries)
#define GS2_TILE_PIX (GS2_TILE * GS2_TILE)
#define GS2_ZPOS 48                  // image-space payload (moments) of the position group, the largest
#define GS2_ZSUM 41                  // the position group's z-space sums rebuilt from it (g, H, cross, colour)
#define GS2_MAX_SH 16

// device status bits
#define GS2_ST_CAPACITY 1u
#define GS2_ST_NONFINITE 2u
#define GS2_ST_TIMEOUT 4u

static inline int sh_count(int deg) { return (deg + 1) * (deg + 1); }

// Sort state of one binning (uint32 words, zeroed at the start of every
// binning): the tiles-touched scan's chunk ticket and its look-back states
// (GS2_SCAN_CHUNKS 64-bit words).
#define GS2_SS_TICKET 0
#define GS2_SS_CHUNKS 2               // 8-byte aligned
#define GS2_SCAN_CHUNKS 256
#define GS2_SS_WORDS (GS2_SS_CHUNKS + 2 * GS2_SCAN_CHUNKS)
// bits of the tile-sort keys 0..ntiles (ntiles marks a dropped pair)
static constexpr int gs2_tile_bits(int64_t ntiles) {
    int bits = 1;
    while ((1ll << bits) <= ntiles) ++bits;
    return bits;
}
static inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// --------------------------------------------------------------------------
// Layout of the caller-owned projection buffer (opaque to callers).
struct ProjView {
    float4 *recA;      // (pi_x, pi_y, conic_xx, conic_xy)
    float4 *recB;      // (conic_yy, sigma, l, lmax): the thresholds of q (decide.cuh)
    float4 *col;       // (c~_r, c~_g, c~_b, ry = padded half height of the support)
    float *k2;         // det Sigma / Sigma_yy^2 (row extent of the support ellipse)
    uint2 *rect;       // tile rectangle: x = tx0 | ty0 << 16, y = tx1 | ty1 << 16 (exclusive ends)
    uint32_t *touched; // tiles of rect that the support ellipse reaches (0 = not rendered)
    uint32_t *key;     // FP32 bit pattern of the camera depth (positive)
    uint32_t *offs;    // exclusive prefix sum of touched, in depth-rank order
    uint32_t *dk[2];   // depth-sort keys (ping-pong)
    uint32_t *dv[2];   // depth-sort values: Gaussian ids, finally in depth-rank order
    uint32_t *tsort;   // touched in depth-rank order
};

static inline size_t proj_bytes_impl(int64_t n) {
    size_t b = 0;
    b += align256(16 * (size_t)n) * 3;
    b += align256(8 * (size_t)n);
    b += align256(4 * (size_t)n) * 9;
    return b;
}

static inline ProjView proj_view(void *base, int64_t n) {
    char *p = (char *)base;
    ProjView v;
    v.recA = (float4 *)p; p += align256(16 * (size_t)n);
    v.recB = (float4 *)p; p += align256(16 * (size_t)n);
    v.col = (float4 *)p; p += align256(16 * (size_t)n);
    v.k2 = (float *)p; p += align256(4 * (size_t)n);
    v.rect = (uint2 *)p; p += align256(8 * (size_t)n);
    v.touched = (uint32_t *)p; p += align256(4 * (size_t)n);
    v.key = (uint32_t *)p; p += align256(4 * (size_t)n);
    v.offs = (uint32_t *)p; p += align256(4 * (size_t)n);
    for (int i = 0; i < 2; ++i) {
        v.dk[i] = (uint32_t *)p; p += align256(4 * (size_t)n);
        v.dv[i] = (uint32_t *)p; p += align256(4 * (size_t)n);
    }
    v.tsort = (uint32_t *)p;
    return v;
}

struct RasterView {
    float *tfinal;   // [H*W] final transmittance
    uint32_t *last;  // [H*W] number of tile-list entries consumed (last contributor + 1)
    // split accumulation (all NULL / 0 when off): the compositing also keeps,
    // at every ck_every list entries of a tile's walk, each pixel's T there
    // and the colour (r, g, b) its entries from there on add, and the tile's
    // walk length (largest `last` of its pixels)
    float4 *ck;                 // [slots][GS2_TILE_PIX]: slot r.x / ck_every + j for list position j ck_every
    uint32_t *tile_maxlast;     // [tiles]
    int ck_every;
};

static inline size_t raster_state_bytes_impl(int w, int h) {
    return align256(4 * (size_t)w * h) * 2;
}

static inline RasterView raster_view(void *base, int w, int h) {
    RasterView r;
    r.tfinal = (float *)base;
    r.last = (uint32_t *)((char *)base + align256(4 * (size_t)w * h));
    r.ck = nullptr;
    r.tile_maxlast = nullptr;
    r.ck_every = 0;
    return r;
}

// camera as passed to kernels (by value)
struct DevCam {
    int w, h;
    float fx, fy, cx, cy;
    float V[12];     // row-major [R | t]
    float o[3];      // camera centre
    float Lx, Ly;    // frustum clamp of tx/tz, ty/tz in the projection Jacobian
};

static inline DevCam make_devcam(const gs2_camera *c) {
    DevCam d;
    d.w = c->width;
    d.h = c->height;
    d.fx = c->fx; d.fy = c->fy; d.cx = c->cx; d.cy = c->cy;
    for (int i = 0; i < 12; ++i) d.V[i] = c->viewmat[i];
    d.Lx = c->clip_x > 0.f ? c->clip_x : 1.3f * (0.5f * (float)c->width) / c->fx;
    d.Ly = c->clip_y > 0.f ? c->clip_y : 1.3f * (0.5f * (float)c->height) / c->fy;
    for (int i = 0; i < 3; ++i) {
        double s = 0;
        for (int j = 0; j < 3; ++j) s -= (double)c->viewmat[j * 4 + i] * (double)c->viewmat[j * 4 + 3];
        d.o[i] = (float)s;
    }
    return d;
}

struct DevScene {
    int n, S;
    const float *mean, *quat, *scale, *opacity, *sh;
};

static inline DevScene make_devscene(const gs2_scene *s) {
    DevScene d;
    d.n = s->n;
    d.S = sh_count(s->sh_degree);
    d.mean = s->mean; d.quat = s->quat; d.scale = s->scale; d.opacity = s->opacity; d.sh = s->sh;
    return d;
}

// --------------------------------------------------------------------------
struct gs2_ctx {
    gs2_config cfg;
    int64_t max_n;
    int max_w, max_h, max_sh;
    int64_t max_pairs;
    int nb_sort;                 // blocks of the radix sort grid (tuning, <= GS2_SORT_BLOCKS_MAX)
    int sort_rows;               // keys per thread per scatter round (tuning: 2, 4, 8 or 16)
    int view_lanes;              // run a sweep's views concurrently (tuning: 0, 1)
    int accum_px;                // pixels per thread of the position accumulation (tuning: 2 or 4)
    int accum_split;             // list entries per work item of the split accumulation (tuning; 0: off)
    // split accumulation: a tile's back-to-front walk cut into items of
    // accum_split entries, each started from the compositing's checkpoint at
    // its back end, fetched by a persistent grid longest tiles first
    float4 *ck;                  // [ck_slots][GS2_TILE_PIX] per-pixel checkpoints (T, C) of the compositing
    size_t ck_slots;
    int ck_ca;                   // accum_split the checkpoints are sized for (smallest allowed)
    uint32_t *tile_maxlast;      // [max tiles] walk length of every tile
    uint4 *acc_items;            // [acc_items_cap] (tile, first entry, end entry, checkpoint slot or ~0)
    size_t acc_items_cap;
    uint32_t *acc_ctrl;          // [0] items, [1] fetch counter
    int rs_split;                // accum_split of the last compositing on this context (0: no checkpoints)
    // sorting
    uint32_t *keys[2];           // pair keys: tile id
    uint32_t *vals[2];           // pair values: Gaussian id
    uint32_t *ghist;             // [256][nb_sort] block histograms of the depth sort
    uint32_t *sort_state;        // GS2_SS_WORDS: the tiles-touched scan's ticket and chunk states
    uint32_t *d_count;           // [0] clamped pair count, [1] raw count, [2] Gaussian count (depth sort),
                                 // [3] listed pairs (the live keys)
    uint2 *ranges;               // [max tiles]
    int sorted;                  // which of keys/vals holds the sorted pairs
    const uint32_t *list_ids;    // Gaussian ids of the sorted tile lists (vals[sorted], or det_list)
    uint32_t *tile_order;        // [max tiles] tiles by descending list length (launch order of the
                                 // compositing and accumulation grids), or NULL: row-major order
    // deterministic mode (cfg.deterministic): per-list-entry partials instead
    // of float atomics, reduced per Gaussian in a fixed order
    float *det_part;             // [max_pairs][GS2_ZPOS] image-space payload of every (tile, Gaussian) entry
    uint32_t *det_ids;           // [max_pairs] Gaussian id of every emitted pair (emission order)
    uint32_t *det_inv;           // [max_pairs] sorted position of every emitted pair
    uint32_t *det_list;          // [max_pairs] Gaussian ids in sorted order
    const uint32_t *det_order;   // depth (rank) order of the last binning
    int tiles_x, tiles_y;        // of the last gs2_raster_fwd
    // accumulation
    float *zbuf;                 // [GS2_ZPOS][max_n], zero between uses
    float *pix_e, *pix_h;        // [3][max_w*max_h]
    // sweep scratch
    void *sw_proj;
    void *sw_rstate;
    float *sw_image;
    float *sw_tgt;               // downsampled secondary targets
    void *sw_blocks;
    void *sw_step;
    size_t sw_blocks_bytes, sw_step_bytes;
    uint32_t *d_status;
    uint8_t *flags;              // [max_n] per-Gaussian flags (FP64 re-solve of the colour block)
    const void *mlp_w;           // installed step-scale network (BF16, caller-owned) or NULL
    const void *damp_w;          // installed damping network (BF16, caller-owned) or NULL
    void *lane_blocks;           // a view lane's own blocks of one view (allocated when a network is
                                 // installed): its epilogue adds there, not into the shared blocks,
                                 // so that the primary view's gradient is copied free of the others'
    float *d_rho;                // [max_n] per-Gaussian damping multipliers of the learned damping
    // logged damping labels (allocated by the first gs2_sweep_logged that asks for them)
    void *lg_bloc;               // the group's local blocks (the views it was solved from)
    void *lg_ball;               // the group's blocks summed (colour: one slot per view) over every training view
    void *lg_step2;              // a candidate step
    float *lg_bq, *lg_brho;      // [max_n] best quadratic-model value so far and its multiplier
    float *lg_wq;                // [max_n] largest finite quadratic-model value so far
    size_t lg_ball_bytes, lg_bloc_bytes;
    float *g_prim;               // [3][max_n] gradient rows right after the view-slot-0 accumulation
    float *lg_phi;               // [max_n] phi1 accumulator of the logged sweep
    uint32_t *order_cache;       // [1 + knn_k][max_n] depth orders of a sweep's views (reused while means are fixed)
    void *jb_mem;                // Jacobi over groups: one allocation holding ...
    float *jb_blocks[5];         // ... every group's blocks (1 + knn_k view slots for colour) and ...
    float *jb_step[5];           // ... every group's step
    // opt-in profile of the accumulation kernel: CUDA events around every launch
    // and per-group pair / visible-Gaussian totals counted on the device
    int prof_on;
    int prof_n;                  // event pairs used in the pool
    cudaEvent_t prof_ev[2 * GS2_PROF_POOL];
    int prof_group[GS2_PROF_POOL];   // 0..4: accumulation of that group; GS2_PROF_BIN/RASTER/LOSS: stages
    unsigned long long *d_stats; // [5][4]: pairs, visible Gaussians, binnings, accumulation evaluations
    unsigned long long *d_resolves; // [5]: blocks (colour: channels) solved again in FP64, per group
    int stat_slot;               // group slot the binning statistics go to
    unsigned long long h_pixels[5];
    std::string err;
    // view lanes: a sweep runs the views of a group concurrently, view slot
    // i >= 1 on lane i - 1 (own sorting / render / accumulation scratch and
    // stream, sharing the status word, the statistics and the depth-order
    // cache); owner: the context whose profile pool and statistics a lane uses
    gs2_ctx *owner;
    int n_lanes;
    gs2_ctx *lanes[GS2_MAX_LANES];
    cudaStream_t lane_st[GS2_MAX_LANES];
    cudaEvent_t lane_ev[GS2_MAX_LANES + 1];
};

// number of kernels this library has launched (host-side count)
extern std::atomic<unsigned long long> g_gs2_launches;
#define GS2_COUNT_LAUNCH(k) (g_gs2_launches.fetch_add((k), std::memory_order_relaxed))

// --------------------------------------------------------------------------
// launchers implemented in the .cu files (return a CUDA error code)
// up to GS2_PROJ_VIEWS views of one scene projected by one launch
#define GS2_PROJ_VIEWS 4
struct ProjViews {
    int nv;
    DevCam cam[GS2_PROJ_VIEWS];
    ProjView pv[GS2_PROJ_VIEWS];
};
cudaError_t launch_project_views(const DevScene &sc, const ProjViews &views, const gs2_config &cfg, cudaStream_t st,
                                 uint32_t *status);
cudaError_t launch_project(const DevScene &sc, const DevCam &cam, const gs2_config &cfg, ProjView pv, int tiles_x,
                           int tiles_y, cudaStream_t st, uint32_t *status);
// order_in: a depth order of the same means and camera to reuse (skips the
// depth sort); order_out: where to keep the computed one (both may be NULL)
cudaError_t launch_debug_lookback(gs2_ctx *ctx, int c, uint32_t limit, cudaStream_t st);
cudaError_t launch_bin_sort(gs2_ctx *ctx, ProjView pv, int n, int tiles_x, int tiles_y, cudaStream_t st,
                            unsigned long long *stats, const uint32_t *order_in = nullptr,
                            uint32_t *order_out = nullptr);
cudaError_t launch_raster(gs2_ctx *ctx, ProjView pv, const DevCam &cam, const gs2_config &cfg, float *image,
                          RasterView rv, cudaStream_t st);
cudaError_t launch_loss(const float *image, const float *target, int w, int h, const gs2_config &cfg, float *e,
                        float *hh, double *loss_out, cudaStream_t st, uint32_t *status);
cudaError_t launch_accum(gs2_ctx *ctx, int group, const DevScene &sc, const DevCam &view, const DevCam &primary,
                         ProjView pv, RasterView rv, const gs2_config &cfg, int view_slot, void *blocks,
                         cudaStream_t st);
// allocates the split accumulation's checkpoints and work items of a context
// (and its view lanes) for chunks of ca list entries (host side, never under
// stream capture); false on allocation failure
bool ensure_split(gs2_ctx *ctx, int ca);
// occupancy of the split accumulation kernels, asked once from the host
void prepare_split_kernels();
// rho: per-Gaussian multiplier of the damping mu0 (the learned damping), or NULL
cudaError_t launch_solve(int group, const void *blocks, int n_views, const DevScene &sc, const DevCam &primary,
                         const gs2_config &cfg, void *step, int32_t *n_failed, uint8_t *flags, cudaStream_t st,
                         unsigned long long *resolves, const float *rho = nullptr);
cudaError_t launch_apply(int group, const void *step, const DevScene &sc, const DevCam &primary,
                         const gs2_config &cfg, cudaStream_t st);
cudaError_t launch_downsample(const float *in, int w, int h, int f, float *out, cudaStream_t st);
cudaError_t prepare_loss_kernels();
// profiling: an event pair around a stage's launches on stream st (no-ops
// unless profiling is on and the pool has room); returns the pair index or -1
int prof_begin(gs2_ctx *ctx, int tag, cudaStream_t st);
void prof_end(gs2_ctx *ctx, int idx, cudaStream_t st);
// validation of a configuration (gs2_create, gs2_set_config, gs2_render_noalloc):
// false with a message in err when a field is out of its range
bool cfg_ok(const gs2_config *c, std::string &err);
// one sweep on ctx (gs2_sweep / gs2_sweep_logged; records may be NULL)
gs2_status sweep_run(gs2_ctx *ctx, gs2_scene *scene, const gs2_camera *cams, int32_t ncam,
                     const float *const *targets, const int32_t *knn, int32_t t, float *records, double *losses_out,
                     int32_t *n_failed, cudaStream_t stream, float *records_damp = nullptr);
cudaError_t launch_step_records(int group, const void *blocks, int n_views, const DevScene &sc, const void *step,
                                const float *gp, const gs2_config &cfg, float *rec, cudaStream_t st);
cudaError_t launch_step_labels(int group, const void *blocks_after, int n_views, const DevScene &sc,
                               const void *step, const float *phi1, float *rec, cudaStream_t st);
cudaError_t launch_phi_add(int group, const void *blocks_one_view, const DevScene &sc, const void *step, float *out,
                           cudaStream_t st);
cudaError_t launch_learned_scale(int group, const void *blocks, int n_views, const DevScene &sc, void *step,
                                 const float *gp, const gs2_config &cfg, const void *w, cudaStream_t st);
// learned damping: the groups whose damping changes the step's direction
__host__ __device__ constexpr bool damping_learned(int group) {
    return group == GS2_POS || group == GS2_SCALE || group == GS2_COLOR;
}
cudaError_t launch_learned_damping(int group, const void *blocks, int n_views, const DevScene &sc, const void *step,
                                   const float *gp, const gs2_config &cfg, const void *w, float *rho,
                                   cudaStream_t st);
cudaError_t launch_damp_eval(int group, const void *blocks_all, int n_all, const DevScene &sc, const void *step,
                             const gs2_config &cfg, float rho_j, float *best_q, float *best_rho, float *worst_q,
                             int first, cudaStream_t st);
cudaError_t launch_damp_labels(int group, const float *rec, const float *best_q, const float *worst_q,
                               const float *best_rho, int n, float *rec_damp, cudaStream_t st);
cudaError_t launch_add_floats(float *dst, const float *src, size_t count, cudaStream_t st);
cudaError_t launch_bounding_sphere(const DevScene &sc, float *out, cudaStream_t st);

// --------------------------------------------------------------------------
// Device helpers shared by the rasteriser and the accumulation: both must take
// the same alpha decisions bit for bit, so the Gaussian falloff is evaluated
// with explicitly rounded operations (no compiler contraction choices).
#ifdef __CUDACC__
// Pixel of thread t in its tile (compositing, one thread per pixel): warp w
// covers the 8x4 block (w % (T/8), w / (T/8)) of the tile, lane l its pixel
// (l % 8, l / 8) -- compact warp blocks keep more of a warp's lanes inside a
// small Gaussian footprint than T x 2 rows do.
#define GS2_WPR (GS2_TILE / 8)       // 8-pixel-wide warp blocks per tile row
__device__ __forceinline__ int gs2_tile_px(int t) { return ((t >> 5) % GS2_WPR) * 8 + (t & 7); }
__device__ __forceinline__ int gs2_tile_py(int t) { return ((t >> 5) / GS2_WPR) * 4 + ((t >> 3) & 3); }

// Two pixels per thread (accumulation, GS2_PAIR_THREADS per tile): warp w
// covers the 8x8 block ((w % (T/8)) 8, (w / (T/8)) 8), lane l the pixels
// (l % 8, l / 8) and (l % 8, l / 8 + 4) of it.  One warp reduction serves
// both pixels of a lane (a Gaussian that reaches one 8x4 half of such a
// block nearly always reaches the other).  The compositing keeps one pixel
// per thread: there a lane would run on until both of its pixels saturate
// (measured slower).
#define GS2_PAIR_THREADS (GS2_TILE_PIX / 2)
#define GS2_PAIR_WARPS (GS2_PAIR_THREADS / 32)
__device__ __forceinline__ int gs2_pair_px(int t) { return ((t >> 5) % GS2_WPR) * 8 + (t & 7); }
__device__ __forceinline__ int gs2_pair_py(int t) { return ((t >> 5) / GS2_WPR) * 8 + ((t >> 3) & 3); }

// asynchronous 16-byte global -> shared copies (the batch staging pipeline)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Gaussian falloff G = exp(-q/2) of a quadratic form q (dec_quad), taken as
// 2^(-q / (2 ln 2)) with the hardware base-2 exponential (relative error
// ~2^-22, flushed to 0 below the normal range: far inside the image and
// derivative tolerances).  It gives the composited values only; whether a term
// is composited or clamped is decided from q itself (decide.cuh), identically
// in the compositing and the accumulation.
__device__ __forceinline__ float gs2_falloff(float q) {
    const float x = __fmul_rn(q, -0.72134752044448170368f);   // -1 / (2 ln 2)
    float g;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(g) : "f"(x));
    return g;
}
#endif
