// C-ABI entry points of libgs2.so: argument checking, scratch ownership and
// launch sequencing.  Every compute step runs in the kernels of this library.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

#define RET_CUDA(ctx, expr)                                                                       \
    do {                                                                                          \
        cudaError_t e_ = (expr);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            if (ctx) (ctx)->err = std::string(#expr) + ": " + cudaGetErrorString(e_);             \
            return GS2_ERR_CUDA;                                                                  \
        }                                                                                         \
    } while (0)

#define REQUIRE(ctx, cond, code, msg)                                                             \
    do {                                                                                          \
        if (!(cond)) {                                                                            \
            if (ctx) (ctx)->err = (msg);                                                          \
            return (code);                                                                        \
        }                                                                                         \
    } while (0)

static const int SORT_BLOCKS = 148 * 4;

std::atomic<unsigned long long> g_gs2_launches{0};

extern "C" void gs2_config_default(gs2_config *c) {
    if (!c) return;
    c->lambda_ssim = 0.2f;
    c->alpha_min = 1.f / 255.f;
    c->alpha_max = 0.99f;
    c->t_min = 1e-4f;
    c->lowpass = 0.3f;
    c->near_z = 0.2f;
    c->barrier_alpha = 1e-6f;
    c->frac_to_boundary = 0.99f;
    c->damping_mu0 = 1.0f;
    c->damping_tries = 6;
    c->scale_min = 1e-7f;
    c->scale_trust = 1.05f;
    c->trust_pos = 0.05f;
    c->trust_rot = 0.05f;
    c->trust_color = 0.05f;
    c->ssim_c1 = 1e-4f;
    c->ssim_c2 = 9e-4f;
    c->ssim_sigma = 1.5f;
    c->ssim_radius = 5;
    c->knn_k = 3;
    c->downsample = 2;
    c->precision = 0;
    c->gauss_newton = 0;
    for (int i = 0; i < 5; ++i) c->group_order[i] = i;
    c->group_jacobi = 0;
    for (int i = 0; i < 5; ++i) c->gd_lr[i] = 0.f;
    c->deterministic = 0;
    c->learned_trust = 1.f;
}

bool cfg_ok(const gs2_config *c, std::string &err) {
    if (!(c->alpha_min > 0.f && c->alpha_min < 1.f)) { err = "alpha_min must be in (0,1)"; return false; }
    if (!(c->alpha_max >= c->alpha_min && c->alpha_max <= 1.f)) { err = "alpha_max must be in [alpha_min,1]"; return false; }
    if (!(c->t_min >= 0.f && c->t_min < 1.f)) { err = "t_min must be in [0,1)"; return false; }
    if (!(c->lowpass >= 0.f) || !(c->near_z > 0.f)) { err = "lowpass >= 0 and near_z > 0 required"; return false; }
    if (c->ssim_radius != 5) { err = "only an 11x11 SSIM window (ssim_radius 5) is supported"; return false; }
    if (c->knn_k < 0 || c->knn_k > 16) { err = "knn_k must be in [0,16]"; return false; }
    if (c->downsample < 1 || c->downsample > 8) { err = "downsample must be in [1,8]"; return false; }
    if (c->damping_tries < 0 || c->damping_tries > 30 || !(c->damping_mu0 >= 0.f)) { err = "bad damping"; return false; }
    if (!(c->scale_trust > 1.f) || !(c->scale_min > 0.f)) { err = "scale_trust > 1 and scale_min > 0 required"; return false; }
    if (!(c->frac_to_boundary > 0.f && c->frac_to_boundary < 1.f)) { err = "frac_to_boundary in (0,1)"; return false; }
    if (!(c->trust_pos > 0.f && c->trust_rot > 0.f && c->trust_color > 0.f)) { err = "trust radii must be > 0"; return false; }
    if (c->gauss_newton != 0 && c->gauss_newton != 1) { err = "gauss_newton must be 0 or 1"; return false; }
    int seen = 0;
    for (int i = 0; i < 5; ++i) {
        if (c->group_order[i] < 0 || c->group_order[i] > 4) { err = "group_order entries must be groups 0..4"; return false; }
        seen |= 1 << c->group_order[i];
    }
    if (seen != 31) { err = "group_order must be a permutation of the five groups"; return false; }
    if (c->group_jacobi != 0 && c->group_jacobi != 1) { err = "group_jacobi must be 0 or 1"; return false; }
    for (int i = 0; i < 5; ++i)
        if (!(c->gd_lr[i] >= 0.f) || !isfinite(c->gd_lr[i])) { err = "gd_lr entries must be finite and >= 0"; return false; }
    if (c->deterministic != 0 && c->deterministic != 1) { err = "deterministic must be 0 or 1"; return false; }
    if (!(c->learned_trust >= 1.f && c->learned_trust <= 16.f)) { err = "learned_trust must be in [1, 16]"; return false; }
    return true;
}

static size_t blocks_bytes_impl(int group, int64_t n, int sh_degree, int n_views) {
    const int S = sh_count(sh_degree);
    switch (group) {
    case GS2_POS:
    case GS2_SCALE: return sizeof(float) * 9 * (size_t)n;
    case GS2_ROT:
    case GS2_OPACITY: return sizeof(float) * 2 * (size_t)n;
    default: return sizeof(float) * (size_t)(6 + S) * n * (size_t)n_views;
    }
}

static size_t step_bytes_impl(int group, int64_t n, int sh_degree) {
    switch (group) {
    case GS2_POS:
    case GS2_SCALE: return sizeof(float) * 3 * (size_t)n;
    case GS2_ROT:
    case GS2_OPACITY: return sizeof(float) * (size_t)n;
    default: return sizeof(float) * 3 * (size_t)sh_count(sh_degree) * n;
    }
}

extern "C" size_t gs2_proj_bytes(int64_t n) { return proj_bytes_impl(n < 1 ? 1 : n); }
extern "C" size_t gs2_raster_state_bytes(int32_t w, int32_t h) { return raster_state_bytes_impl(w, h); }
extern "C" size_t gs2_blocks_bytes(gs2_group g, int64_t n, int32_t sh, int32_t nv) {
    return blocks_bytes_impl(g, n, sh, nv < 1 ? 1 : nv);
}
extern "C" size_t gs2_step_bytes(gs2_group g, int64_t n, int32_t sh) { return step_bytes_impl(g, n, sh); }

// a view lane's own scratch (the rest is shared with its owner)
static void free_lane(gs2_ctx *l) {
    void *ptrs[] = {l->keys[0], l->keys[1], l->vals[0], l->vals[1], l->ghist, l->sort_state, l->d_count, l->ranges,
                    l->zbuf, l->pix_e, l->pix_h, l->sw_proj, l->sw_rstate, l->sw_image, l->tile_order,
                    l->lane_blocks, l->ck, l->tile_maxlast, l->acc_items, l->acc_ctrl};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

static void free_ctx(gs2_ctx *c) {
    for (int i = 0; i < c->n_lanes; ++i) {
        if (c->lanes[i]) {
            free_lane(c->lanes[i]);
            delete c->lanes[i];
        }
        if (c->lane_st[i]) cudaStreamDestroy(c->lane_st[i]);
    }
    for (int i = 0; i <= c->n_lanes && i <= GS2_MAX_LANES; ++i)
        if (c->lane_ev[i]) cudaEventDestroy(c->lane_ev[i]);
    void *ptrs[] = {c->keys[0], c->keys[1], c->vals[0], c->vals[1], c->ghist, c->sort_state, c->d_count, c->ranges,
                    c->zbuf, c->pix_e, c->pix_h, c->sw_proj, c->sw_rstate, c->sw_image, c->sw_tgt, c->sw_blocks,
                    c->sw_step, c->d_status, c->d_stats, c->d_resolves, c->flags, c->g_prim, c->lg_phi,
                    c->d_rho, c->lg_bloc, c->lg_ball, c->lg_step2, c->lg_bq, c->lg_brho, c->lg_wq,
                    c->order_cache, c->jb_mem, c->det_part, c->det_ids, c->det_inv, c->det_list, c->tile_order,
                    c->ck, c->tile_maxlast, c->acc_items, c->acc_ctrl};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->prof_on >= 0 && c->prof_ev[0])
        for (int i = 0; i < 2 * GS2_PROF_POOL; ++i)
            if (c->prof_ev[i]) cudaEventDestroy(c->prof_ev[i]);
}

// split accumulation buffers of one context, sized for chunks of ca entries
// (any larger chunk fits: fewer checkpoint slots and items)
static bool split_buffers(gs2_ctx *c, int ca) {
    if (c->ck && c->ck_ca <= ca) return true;
    if (cudaDeviceSynchronize() != cudaSuccess) return false;   // the old buffers may be in use
    void *old[] = {c->ck, c->tile_maxlast, c->acc_items, c->acc_ctrl};
    for (void *p : old)
        if (p) cudaFree(p);
    c->ck = nullptr;
    c->tile_maxlast = nullptr;
    c->acc_items = nullptr;
    c->acc_ctrl = nullptr;
    c->ck_ca = 0;
    c->rs_split = 0;
    const size_t tiles = (size_t)((c->max_w + GS2_TILE - 1) / GS2_TILE) * ((c->max_h + GS2_TILE - 1) / GS2_TILE);
    const size_t pairs = (size_t)std::max<int64_t>(c->max_pairs, 1);
    c->ck_slots = (pairs - 1) / (size_t)ca + 1;
    c->acc_items_cap = tiles + pairs / (size_t)ca + 1;
    bool ok = cudaMalloc((void **)&c->ck, sizeof(float4) * GS2_TILE_PIX * c->ck_slots) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&c->tile_maxlast, sizeof(uint32_t) * tiles) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&c->acc_items, sizeof(uint4) * c->acc_items_cap) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&c->acc_ctrl, sizeof(uint32_t) * 2) == cudaSuccess;
    ok = ok && cudaMemset(c->acc_ctrl, 0, sizeof(uint32_t) * 2) == cudaSuccess;
    if (!ok) {
        void *got[] = {c->ck, c->tile_maxlast, c->acc_items, c->acc_ctrl};
        for (void *p : got)
            if (p) cudaFree(p);
        c->ck = nullptr;
        c->tile_maxlast = nullptr;
        c->acc_items = nullptr;
        c->acc_ctrl = nullptr;
        return false;
    }
    c->ck_ca = ca;
    return true;
}

bool ensure_split(gs2_ctx *ctx, int ca) {
    if (ca <= 0) return true;
    prepare_split_kernels();
    if (!split_buffers(ctx, ca)) return false;
    for (int i = 0; i < ctx->n_lanes; ++i)
        if (ctx->lanes[i] && !split_buffers(ctx->lanes[i], ca)) return false;
    return true;
}

// Jacobi over groups: every group's blocks and step at once (allocated when
// the option is first set, from the host, never inside a stream capture)
static bool ensure_jacobi(gs2_ctx *c) {
    if (c->jb_mem) return true;
    const int K = c->cfg.knn_k;
    size_t off[11], tot = 0;
    for (int g = 0; g < 5; ++g) {
        off[g] = tot;
        tot += align256(blocks_bytes_impl(g, c->max_n, c->max_sh, 1 + K));
    }
    for (int g = 0; g < 5; ++g) {
        off[5 + g] = tot;
        tot += align256(step_bytes_impl(g, c->max_n, c->max_sh));
    }
    if (cudaMalloc(&c->jb_mem, tot) != cudaSuccess) {
        c->jb_mem = nullptr;
        return false;
    }
    for (int g = 0; g < 5; ++g) {
        c->jb_blocks[g] = (float *)((char *)c->jb_mem + off[g]);
        c->jb_step[g] = (float *)((char *)c->jb_mem + off[5 + g]);
    }
    return true;
}

// deterministic mode: the per-entry partials and the index arrays (allocated
// when the option is first set, from the host, never inside a stream capture)
static bool ensure_det(gs2_ctx *c) {
    if (c->det_part) return true;
    const size_t M = (size_t)c->max_pairs;
    void *p[4] = {nullptr, nullptr, nullptr, nullptr};
    const size_t bytes[4] = {sizeof(float) * GS2_ZPOS * M, sizeof(uint32_t) * M, sizeof(uint32_t) * M,
                             sizeof(uint32_t) * M};
    for (int i = 0; i < 4; ++i)
        if (cudaMalloc(&p[i], bytes[i]) != cudaSuccess) {
            for (int j = 0; j < 4; ++j)
                if (p[j]) cudaFree(p[j]);
            cudaGetLastError();
            return false;
        }
    c->det_part = (float *)p[0];
    c->det_ids = (uint32_t *)p[1];
    c->det_inv = (uint32_t *)p[2];
    c->det_list = (uint32_t *)p[3];
    return true;
}

extern "C" gs2_status gs2_create(gs2_ctx **out, const gs2_config *cfg, int64_t max_n, int32_t max_w, int32_t max_h,
                                 int32_t max_sh, int64_t max_pairs) {
    if (!out) return GS2_ERR_ARG;
    *out = nullptr;
    if (max_n < 1 || max_w < 1 || max_h < 1 || max_sh < 0) return GS2_ERR_ARG;
    if (max_sh > 3) return GS2_ERR_UNSUPPORTED;
    if (max_n > (int64_t)0x7FFFFFFF || (int64_t)max_w * max_h > (int64_t)1 << 28) return GS2_ERR_SHAPE;
    // tile rectangles hold 16-bit tile coordinates
    if (max_w > 0xFFFF * GS2_TILE || max_h > 0xFFFF * GS2_TILE) return GS2_ERR_SHAPE;
    gs2_ctx *c = new (std::nothrow) gs2_ctx();
    if (!c) return GS2_ERR_OOM;
    if (cfg) c->cfg = *cfg;
    else gs2_config_default(&c->cfg);
    if (!cfg_ok(&c->cfg, c->err)) {
        delete c;
        return GS2_ERR_ARG;
    }
    if (prepare_loss_kernels() != cudaSuccess) {
        delete c;
        cudaGetLastError();
        return GS2_ERR_CUDA;
    }
    if (max_pairs <= 0) max_pairs = 16 * max_n;
    if (max_pairs > (int64_t)0xF0000000ll) max_pairs = (int64_t)0xF0000000ll;
    c->max_n = max_n;
    c->max_w = max_w;
    c->max_h = max_h;
    c->max_sh = max_sh;
    c->max_pairs = max_pairs;
    c->nb_sort = SORT_BLOCKS;
    c->sort_rows = 4;
    c->view_lanes = 1;
    c->accum_px = GS2_TILE == 16 ? 4 : 2;   // measured: position accumulation 3.77 -> 3.20 ms per sweep
    const size_t P = (size_t)max_w * max_h;
    const int tiles = ((max_w + GS2_TILE - 1) / GS2_TILE) * ((max_h + GS2_TILE - 1) / GS2_TILE);
    const int K = c->cfg.knn_k, f = c->cfg.downsample;
    const int S = sh_count(max_sh);
    bool ok = true;
    auto A = [&](void **p, size_t bytes) {
        if (!ok) return;
        if (cudaMalloc(p, bytes < 256 ? 256 : bytes) != cudaSuccess) {
            ok = false;
            *p = nullptr;
        }
    };
    for (int i = 0; i < 2; ++i) {
        A((void **)&c->keys[i], sizeof(uint32_t) * (size_t)max_pairs);
        A((void **)&c->vals[i], sizeof(uint32_t) * (size_t)max_pairs);
    }
    A((void **)&c->ghist, sizeof(uint32_t) * (256 * (size_t)GS2_SORT_BLOCKS_MAX + 256));  // + digit totals
    A((void **)&c->sort_state, sizeof(uint32_t) * GS2_SS_WORDS);
    A((void **)&c->d_count, sizeof(uint32_t) * 4);
    A((void **)&c->ranges, sizeof(uint2) * (size_t)tiles);
    A((void **)&c->tile_order, sizeof(uint32_t) * (size_t)tiles);
    A((void **)&c->zbuf, sizeof(double) * GS2_ZPOS * (size_t)max_n);   // FP64 with precision = 1
    A((void **)&c->pix_e, sizeof(float) * 3 * P);
    A((void **)&c->pix_h, sizeof(float) * 3 * P);
    A(&c->sw_proj, proj_bytes_impl(max_n));
    A(&c->sw_rstate, raster_state_bytes_impl(max_w, max_h));
    A((void **)&c->sw_image, sizeof(float) * 3 * P);
    A((void **)&c->sw_tgt, sizeof(float) * 3 * (size_t)(max_w / f) * (max_h / f) * (size_t)std::max(K, 1));
    size_t bmax = 0;
    for (int g = 0; g < 5; ++g) bmax = std::max(bmax, blocks_bytes_impl(g, max_n, max_sh, 1 + K));
    c->sw_blocks_bytes = bmax;
    A(&c->sw_blocks, bmax);
    c->sw_step_bytes = sizeof(float) * 3 * (size_t)S * max_n;
    A(&c->sw_step, c->sw_step_bytes);
    A((void **)&c->d_status, sizeof(uint32_t) * 4);
    A((void **)&c->d_stats, sizeof(unsigned long long) * 5 * 5);
    A((void **)&c->d_resolves, sizeof(unsigned long long) * 5);
    A((void **)&c->flags, (size_t)max_n);
    A((void **)&c->g_prim, sizeof(float) * 3 * (size_t)max_n);
    A((void **)&c->lg_phi, sizeof(float) * (size_t)max_n);
    A((void **)&c->d_rho, sizeof(float) * (size_t)max_n);
    A((void **)&c->order_cache, sizeof(uint32_t) * (size_t)(1 + K) * max_n);
    if (ok) ok = cudaMemset(c->zbuf, 0, sizeof(double) * GS2_ZPOS * (size_t)max_n) == cudaSuccess;
    if (ok) ok = cudaMemset(c->d_status, 0, sizeof(uint32_t) * 4) == cudaSuccess;
    if (ok) ok = cudaMemset(c->d_count, 0, sizeof(uint32_t) * 4) == cudaSuccess;
    if (ok) ok = cudaMemset(c->d_stats, 0, sizeof(unsigned long long) * 25) == cudaSuccess;
    if (ok) ok = cudaMemset(c->d_resolves, 0, sizeof(unsigned long long) * 5) == cudaSuccess;
    // view lanes for the secondaries of a sweep
    c->owner = nullptr;
    c->n_lanes = 0;
    const int nl = std::min(K, GS2_MAX_LANES);
    for (int i = 0; i < nl && ok; ++i) {
        gs2_ctx *l = new (std::nothrow) gs2_ctx();
        if (!l) {
            ok = false;
            break;
        }
        c->lanes[i] = l;
        c->n_lanes = i + 1;
        l->cfg = c->cfg;
        l->max_n = max_n;
        l->max_w = max_w;
        l->max_h = max_h;
        l->max_sh = max_sh;
        l->max_pairs = max_pairs;
        l->nb_sort = c->nb_sort;
        l->sort_rows = c->sort_rows;
        l->accum_px = c->accum_px;
        for (int j = 0; j < 2; ++j) {
            A((void **)&l->keys[j], sizeof(uint32_t) * (size_t)max_pairs);
            A((void **)&l->vals[j], sizeof(uint32_t) * (size_t)max_pairs);
        }
        A((void **)&l->ghist, sizeof(uint32_t) * (256 * (size_t)GS2_SORT_BLOCKS_MAX + 256));
        A((void **)&l->sort_state, sizeof(uint32_t) * GS2_SS_WORDS);
        A((void **)&l->d_count, sizeof(uint32_t) * 4);
        A((void **)&l->ranges, sizeof(uint2) * (size_t)tiles);
        A((void **)&l->tile_order, sizeof(uint32_t) * (size_t)tiles);
        A((void **)&l->zbuf, sizeof(double) * GS2_ZPOS * (size_t)max_n);
        A((void **)&l->pix_e, sizeof(float) * 3 * P);
        A((void **)&l->pix_h, sizeof(float) * 3 * P);
        A(&l->sw_proj, proj_bytes_impl(max_n));
        A(&l->sw_rstate, raster_state_bytes_impl(max_w, max_h));
        A((void **)&l->sw_image, sizeof(float) * 3 * P);
        if (ok) ok = cudaMemset(l->zbuf, 0, sizeof(double) * GS2_ZPOS * (size_t)max_n) == cudaSuccess;
        if (ok) ok = cudaMemset(l->d_count, 0, sizeof(uint32_t) * 4) == cudaSuccess;
        l->d_status = c->d_status;
        l->d_stats = c->d_stats;
        l->d_resolves = c->d_resolves;
        l->order_cache = c->order_cache;
        l->owner = c;
        if (ok) ok = cudaStreamCreateWithFlags(&c->lane_st[i], cudaStreamNonBlocking) == cudaSuccess;
    }
    for (int i = 0; i <= nl && ok; ++i)
        ok = cudaEventCreateWithFlags(&c->lane_ev[i], cudaEventDisableTiming) == cudaSuccess;
    if (ok && c->cfg.group_jacobi) ok = ensure_jacobi(c);
    if (ok && c->cfg.deterministic) ok = ensure_det(c);
    if (!ok) {
        free_ctx(c);
        delete c;
        cudaGetLastError();
        return GS2_ERR_OOM;
    }
    *out = c;
    return GS2_OK;
}

extern "C" gs2_status gs2_destroy(gs2_ctx *ctx) {
    if (!ctx) return GS2_ERR_ARG;
    free_ctx(ctx);
    delete ctx;
    return GS2_OK;
}

extern "C" const char *gs2_last_error(const gs2_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" gs2_status gs2_set_config(gs2_ctx *ctx, const gs2_config *cfg) {
    if (!ctx || !cfg) return GS2_ERR_ARG;
    std::string err;
    REQUIRE(ctx, cfg_ok(cfg, err), GS2_ERR_ARG, err);
    REQUIRE(ctx, cfg->knn_k <= ctx->cfg.knn_k || cfg->knn_k == 0, GS2_ERR_SHAPE,
            "knn_k larger than at gs2_create (sweep scratch sized for it)");
    REQUIRE(ctx, cfg->downsample >= ctx->cfg.downsample, GS2_ERR_SHAPE,
            "downsample smaller than at gs2_create (sweep scratch sized for it)");
    const int K0 = ctx->cfg.knn_k, f0 = ctx->cfg.downsample;
    if (cfg->group_jacobi && !ctx->jb_mem) {
        const gs2_config keep = ctx->cfg;
        ctx->cfg.knn_k = K0;   // sized for the knn_k of gs2_create, like the other sweep scratch
        REQUIRE(ctx, ensure_jacobi(ctx), GS2_ERR_OOM, "cannot allocate the per-group blocks of group_jacobi");
        ctx->cfg = keep;
    }
    if (cfg->deterministic && !ctx->det_part)
        REQUIRE(ctx, ensure_det(ctx), GS2_ERR_OOM, "cannot allocate the partials of deterministic mode");
    ctx->cfg = *cfg;
    ctx->cfg.knn_k = cfg->knn_k;
    (void)K0;
    (void)f0;
    return GS2_OK;
}

extern "C" gs2_status gs2_check(gs2_ctx *ctx, gs2_stream stream) {
    if (!ctx) return GS2_ERR_ARG;
    RET_CUDA(ctx, cudaStreamSynchronize((cudaStream_t)stream));
    uint32_t st = 0;
    RET_CUDA(ctx, cudaMemcpy(&st, ctx->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    RET_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(uint32_t)));
    if (st & GS2_ST_CAPACITY) {
        ctx->err = "more (tile, Gaussian) pairs than max_pairs";
        return GS2_ERR_CAPACITY;
    }
    if (st & GS2_ST_NONFINITE) return GS2_ERR_NONFINITE;
    if (st & GS2_ST_TIMEOUT) return GS2_ERR_TIMEOUT;
    return GS2_OK;
}

static gs2_status check_scene(gs2_ctx *ctx, const gs2_scene *s) {
    REQUIRE(ctx, s != nullptr, GS2_ERR_ARG, "scene is null");
    REQUIRE(ctx, s->n >= 0 && s->n <= ctx->max_n, GS2_ERR_SHAPE, "scene larger than max_gaussians");
    REQUIRE(ctx, s->sh_degree >= 0 && s->sh_degree <= ctx->max_sh, GS2_ERR_SHAPE, "sh_degree above max_sh_degree");
    REQUIRE(ctx, s->n == 0 || (s->mean && s->quat && s->scale && s->opacity && s->sh), GS2_ERR_ARG,
            "scene has a null buffer");
    return GS2_OK;
}

static gs2_status check_cam(gs2_ctx *ctx, const gs2_camera *c) {
    REQUIRE(ctx, c != nullptr, GS2_ERR_ARG, "camera is null");
    REQUIRE(ctx, c->width >= 1 && c->height >= 1, GS2_ERR_ARG, "camera has no pixels");
    REQUIRE(ctx, c->width <= ctx->max_w && c->height <= ctx->max_h, GS2_ERR_SHAPE, "camera larger than max size");
    REQUIRE(ctx, c->fx > 0.f && c->fy > 0.f, GS2_ERR_ARG, "focal lengths must be positive");
    return GS2_OK;
}

#define TRY(x)                        \
    do {                              \
        gs2_status s_ = (x);          \
        if (s_ != GS2_OK) return s_;  \
    } while (0)

static gs2_status do_project(gs2_ctx *ctx, const gs2_scene *scene, const gs2_camera *cam, void *proj,
                             cudaStream_t st) {
    const DevScene sc = make_devscene(scene);
    const DevCam dc = make_devcam(cam);
    const int tx = (cam->width + GS2_TILE - 1) / GS2_TILE, ty = (cam->height + GS2_TILE - 1) / GS2_TILE;
    RET_CUDA(ctx, launch_project(sc, dc, ctx->cfg, proj_view(proj, scene->n), tx, ty, st, ctx->d_status));
    return GS2_OK;
}

extern "C" gs2_status gs2_project(gs2_ctx *ctx, const gs2_scene *scene, const gs2_camera *cam, void *proj,
                                  gs2_stream stream) {
    if (!ctx) return GS2_ERR_ARG;
    TRY(check_scene(ctx, scene));
    TRY(check_cam(ctx, cam));
    REQUIRE(ctx, proj != nullptr, GS2_ERR_ARG, "proj is null");
    return do_project(ctx, scene, cam, proj, (cudaStream_t)stream);
}

static gs2_status do_raster(gs2_ctx *ctx, int n, const gs2_camera *cam, const void *proj, float *image,
                            void *rstate, cudaStream_t st, const uint32_t *order_in = nullptr,
                            uint32_t *order_out = nullptr) {
    ctx->tiles_x = (cam->width + GS2_TILE - 1) / GS2_TILE;
    ctx->tiles_y = (cam->height + GS2_TILE - 1) / GS2_TILE;
    ProjView pv = proj_view(const_cast<void *>(proj), n);
    gs2_ctx *pc = ctx->owner ? ctx->owner : ctx;   // statistics (shared by a sweep's view lanes)
    int pe = prof_begin(ctx, GS2_PROF_BIN, st);
    RET_CUDA(ctx, launch_bin_sort(ctx, pv, n, ctx->tiles_x, ctx->tiles_y, st,
                                  pc->prof_on ? pc->d_stats + 5 * pc->stat_slot : nullptr, order_in, order_out));
    prof_end(ctx, pe, st);
    if (pc->prof_on) pc->h_pixels[pc->stat_slot] += (unsigned long long)cam->width * cam->height;
    pe = prof_begin(ctx, GS2_PROF_RASTER, st);
    RasterView rv = raster_view(rstate, cam->width, cam->height);
    // split accumulation: checkpoints and walk lengths for the accumulations
    // that follow (not in deterministic mode, which walks whole tiles)
    ctx->rs_split = 0;
    if (ctx->accum_split > 0 && ctx->ck && ctx->accum_split >= ctx->ck_ca && !ctx->cfg.deterministic) {
        rv.ck = ctx->ck;
        rv.tile_maxlast = ctx->tile_maxlast;
        rv.ck_every = ctx->accum_split;
        ctx->rs_split = ctx->accum_split;
    }
    RET_CUDA(ctx, launch_raster(ctx, pv, make_devcam(cam), ctx->cfg, image, rv, st));
    prof_end(ctx, pe, st);
    return GS2_OK;
}

extern "C" gs2_status gs2_raster_fwd(gs2_ctx *ctx, const gs2_scene *scene, const gs2_camera *cam, const void *proj,
                                     float *image, void *raster_state, gs2_stream stream) {
    if (!ctx) return GS2_ERR_ARG;
    TRY(check_scene(ctx, scene));
    TRY(check_cam(ctx, cam));
    REQUIRE(ctx, proj && image && raster_state, GS2_ERR_ARG, "null buffer");
    return do_raster(ctx, scene->n, cam, proj, image, raster_state, (cudaStream_t)stream);
}

extern "C" gs2_status gs2_loss_derivs(gs2_ctx *ctx, const float *image, const float *target, int32_t w, int32_t h,
                                      float *e, float *hh, double *loss_out, gs2_stream stream) {
    if (!ctx) return GS2_ERR_ARG;
    REQUIRE(ctx, image && target && e && hh, GS2_ERR_ARG, "null buffer");
    REQUIRE(ctx, w >= 1 && h >= 1, GS2_ERR_ARG, "empty image");
    RET_CUDA(ctx, launch_loss(image, target, w, h, ctx->cfg, e, hh, loss_out, (cudaStream_t)stream, ctx->d_status));
    return GS2_OK;
}

// keep_primary: after a view-slot-0 accumulation, copy the gradient rows into
// ctx->g_prim (the primary view's own gradient, a step-model feature; colour
// keeps it in slot 0 of its blocks)
static gs2_status do_accum(gs2_ctx *ctx, int group, const gs2_scene *scene, const gs2_camera *view,
                           const gs2_camera *primary, const void *proj, const void *rstate, const float *image,
                           const float *target, int slot, void *blocks, double *loss_out, cudaStream_t st,
                           bool keep_primary = true) {
    const int pe = prof_begin(ctx, GS2_PROF_LOSS, st);
    RET_CUDA(ctx, launch_loss(image, target, view->width, view->height, ctx->cfg, ctx->pix_e, ctx->pix_h, loss_out,
                              st, ctx->d_status));
    prof_end(ctx, pe, st);
    RET_CUDA(ctx, launch_accum(ctx, group, make_devscene(scene), make_devcam(view), make_devcam(primary),
                               proj_view(const_cast<void *>(proj), scene->n),
                               raster_view(const_cast<void *>(rstate), view->width, view->height), ctx->cfg, slot,
                               blocks, st));
    if (keep_primary && slot == 0 && group != GS2_COLOR && scene->n > 0) {
        const size_t D = (group == GS2_POS || group == GS2_SCALE) ? 3 : 1;
        RET_CUDA(ctx, cudaMemcpyAsync(ctx->g_prim, blocks, sizeof(float) * D * scene->n, cudaMemcpyDeviceToDevice,
                                      st));
    }
    return GS2_OK;
}

extern "C" gs2_status gs2_accum_newton_blocks(gs2_ctx *ctx, gs2_group group, const gs2_scene *scene,
                                              const gs2_camera *view, const gs2_camera *primary, const void *proj,
                                              const void *raster_state, const float *image, const float *target,
                                              int32_t view_slot, void *blocks, double *loss_out,
                                              gs2_stream stream) {
    if (!ctx) return GS2_ERR_ARG;
    REQUIRE(ctx, group >= GS2_POS && group <= GS2_COLOR, GS2_ERR_ARG, "bad group");
    TRY(check_scene(ctx, scene));
    TRY(check_cam(ctx, view));
    TRY(check_cam(ctx, primary));
    REQUIRE(ctx, proj && raster_state && image && target && blocks, GS2_ERR_ARG, "null buffer");
    REQUIRE(ctx, view_slot >= 0, GS2_ERR_ARG, "negative view_slot");
    REQUIRE(ctx, ctx->tiles_x == (view->width + GS2_TILE - 1) / GS2_TILE &&
                     ctx->tiles_y == (view->height + GS2_TILE - 1) / GS2_TILE,
            GS2_ERR_ARG, "the last gs2_raster_fwd on this context was for a different image size");
    return do_accum(ctx, group, scene, view, primary, proj, raster_state, image, target, view_slot, blocks, loss_out,
                    (cudaStream_t)stream);
}

// The plain damped solve, then the installed networks: the damping network
// (position, scaling, colour) solves again with its per-Gaussian multiplier of
// mu0, the step-scale network scales the result.  With a damping network the
// plain solve counts neither failures nor FP64 re-solves (the second one does).
gs2_status solve_learned(gs2_ctx *ctx, int group, const void *blocks, int n_views, const gs2_scene *scene,
                         const gs2_camera *primary, void *step, int32_t *n_failed, cudaStream_t st) {
    const DevScene dsc = make_devscene(scene);
    const DevCam pc = make_devcam(primary);
    const bool damp = ctx->damp_w && damping_learned(group) && ctx->cfg.gd_lr[group] <= 0.f;
    RET_CUDA(ctx, launch_solve(group, blocks, n_views, dsc, pc, ctx->cfg, step, damp ? nullptr : n_failed, ctx->flags,
                               st, damp ? nullptr : ctx->d_resolves));
    if (damp) {
        RET_CUDA(ctx, launch_learned_damping(group, blocks, n_views, dsc, step, ctx->g_prim, ctx->cfg, ctx->damp_w,
                                             ctx->d_rho, st));
        RET_CUDA(ctx, launch_solve(group, blocks, n_views, dsc, pc, ctx->cfg, step, n_failed, ctx->flags, st,
                                   ctx->d_resolves, ctx->d_rho));
    }
    RET_CUDA(ctx, launch_learned_scale(group, blocks, n_views, dsc, step, ctx->g_prim, ctx->cfg, ctx->mlp_w, st));
    return GS2_OK;
}

extern "C" gs2_status gs2_solve_step(gs2_ctx *ctx, gs2_group group, const void *blocks, int32_t n_views,
                                     const gs2_scene *scene, const gs2_camera *primary, void *step, int32_t *n_failed,
                                     gs2_stream stream) {
    if (!ctx) return GS2_ERR_ARG;
    REQUIRE(ctx, group >= GS2_POS && group <= GS2_COLOR, GS2_ERR_ARG, "bad group");
    TRY(check_scene(ctx, scene));
    TRY(check_cam(ctx, primary));
    REQUIRE(ctx, blocks && step, GS2_ERR_ARG, "null buffer");
    REQUIRE(ctx, n_views >= 1, GS2_ERR_ARG, "n_views must be >= 1");
    TRY(solve_learned(ctx, group, blocks, n_views, scene, primary, step, n_failed, (cudaStream_t)stream));
    return GS2_OK;
}

// With a network installed, a sweep's view lanes add their epilogues into
// blocks of their own (the primary's gradient, a network feature, is then
// copied before any secondary contributes); allocated here, from the host.
static gs2_status ensure_lane_blocks(gs2_ctx *ctx) {
    const size_t bytes = blocks_bytes_impl(GS2_POS, ctx->max_n, ctx->max_sh, 1);   // the largest non-colour block
    for (int i = 0; i < ctx->n_lanes; ++i) {
        gs2_ctx *l = ctx->lanes[i];
        if (l && !l->lane_blocks) RET_CUDA(ctx, cudaMalloc(&l->lane_blocks, bytes));
    }
    return GS2_OK;
}

extern "C" gs2_status gs2_set_damping_model(gs2_ctx *ctx, const uint16_t *w_bf16) {
    if (!ctx) return GS2_ERR_ARG;
    if (w_bf16) TRY(ensure_lane_blocks(ctx));
    ctx->damp_w = w_bf16;
    return GS2_OK;
}

extern "C" gs2_status gs2_set_step_model(gs2_ctx *ctx, const uint16_t *w_bf16) {
    if (!ctx) return GS2_ERR_ARG;
    if (w_bf16) TRY(ensure_lane_blocks(ctx));
    ctx->mlp_w = w_bf16;
    return GS2_OK;
}

static gs2_status check_records_args(gs2_ctx *ctx, int group, const void *blocks, int n_views,
                                     const gs2_scene *scene, const void *step, const float *records) {
    REQUIRE(ctx, group >= GS2_POS && group <= GS2_COLOR, GS2_ERR_ARG, "bad group");
    TRY(check_scene(ctx, scene));
    REQUIRE(ctx, blocks && step && records, GS2_ERR_ARG, "null buffer");
    REQUIRE(ctx, n_views >= 1, GS2_ERR_ARG, "n_views must be >= 1");
    return GS2_OK;
}

extern "C" gs2_status gs2_step_records(gs2_ctx *ctx, gs2_group group, const void *blocks, int32_t n_views,
                                       const gs2_scene *scene, const void *step, float *records, gs2_stream stream) {
    if (!ctx) return GS2_ERR_ARG;
    TRY(check_records_args(ctx, group, blocks, n_views, scene, step, records));
    RET_CUDA(ctx, launch_step_records(group, blocks, n_views, make_devscene(scene), step, ctx->g_prim, ctx->cfg,
                                      records, (cudaStream_t)stream));
    return GS2_OK;
}

extern "C" gs2_status gs2_step_labels(gs2_ctx *ctx, gs2_group group, const void *blocks_after, int32_t n_views,
                                      const gs2_scene *scene, const void *step, float *records, gs2_stream stream) {
    if (!ctx) return GS2_ERR_ARG;
    TRY(check_records_args(ctx, group, blocks_after, n_views, scene, step, records));
    RET_CUDA(ctx, launch_step_labels(group, blocks_after, n_views, make_devscene(scene), step, nullptr, records,
                                     (cudaStream_t)stream));
    return GS2_OK;
}

extern "C" gs2_status gs2_apply_step(gs2_ctx *ctx, gs2_group group, const void *step, gs2_scene *scene,
                                     const gs2_camera *primary, gs2_stream stream) {
    if (!ctx) return GS2_ERR_ARG;
    REQUIRE(ctx, group >= GS2_POS && group <= GS2_COLOR, GS2_ERR_ARG, "bad group");
    TRY(check_scene(ctx, scene));
    TRY(check_cam(ctx, primary));
    REQUIRE(ctx, step != nullptr, GS2_ERR_ARG, "step is null");
    RET_CUDA(ctx, launch_apply(group, step, make_devscene(scene), make_devcam(primary), ctx->cfg,
                               (cudaStream_t)stream));
    return GS2_OK;
}

extern "C" void gs2_camera_downsample(const gs2_camera *in, int32_t f, gs2_camera *out) {
    if (!in || !out || f < 1) return;
    *out = *in;
    out->width = in->width / f;
    out->height = in->height / f;
    out->fx = in->fx / (float)f;
    out->fy = in->fy / (float)f;
    out->cx = (in->cx + 0.5f) / (float)f - 0.5f;
    out->cy = (in->cy + 0.5f) / (float)f - 0.5f;
}

extern "C" gs2_status gs2_downsample(gs2_ctx *ctx, const float *in, int32_t w, int32_t h, int32_t f, float *out,
                                     gs2_stream stream) {
    if (!ctx) return GS2_ERR_ARG;
    REQUIRE(ctx, in && out && f >= 1 && w >= f && h >= f, GS2_ERR_ARG, "bad downsample arguments");
    RET_CUDA(ctx, launch_downsample(in, w, h, f, out, (cudaStream_t)stream));
    return GS2_OK;
}

extern "C" gs2_status gs2_bounding_sphere(gs2_ctx *ctx, const gs2_scene *scene, float *sphere_out,
                                          gs2_stream stream) {
    if (!ctx) return GS2_ERR_ARG;
    TRY(check_scene(ctx, scene));
    REQUIRE(ctx, sphere_out != nullptr && scene->n > 0, GS2_ERR_ARG, "empty scene or null output");
    RET_CUDA(ctx, launch_bounding_sphere(make_devscene(scene), sphere_out, (cudaStream_t)stream));
    return GS2_OK;
}

extern "C" gs2_status gs2_camera_knn(const float *centres, int32_t ncam, const float *sphere, int32_t k,
                                     int32_t *out) {
    if (!centres || !sphere || !out || ncam < 1 || k < 0) return GS2_ERR_ARG;
    std::vector<double> u(3 * (size_t)ncam);
    for (int i = 0; i < ncam; ++i) {
        double nn = 0;
        for (int a = 0; a < 3; ++a) {
            u[i * 3 + a] = (double)centres[i * 3 + a] - (double)sphere[a];
            nn += u[i * 3 + a] * u[i * 3 + a];
        }
        nn = sqrt(nn);
        if (!(nn > 0)) return GS2_ERR_ARG;
        for (int a = 0; a < 3; ++a) u[i * 3 + a] /= nn;
    }
    std::vector<std::pair<double, int>> d;
    for (int i = 0; i < ncam; ++i) {
        d.clear();
        for (int j = 0; j < ncam; ++j) {
            if (j == i) continue;
            double c = u[i * 3] * u[j * 3] + u[i * 3 + 1] * u[j * 3 + 1] + u[i * 3 + 2] * u[j * 3 + 2];
            c = std::min(1.0, std::max(-1.0, c));
            d.emplace_back((double)sphere[3] * acos(c), j);
        }
        std::sort(d.begin(), d.end());
        for (int q = 0; q < k; ++q) out[i * k + q] = q < (int)d.size() ? d[q].second : -1;
    }
    return GS2_OK;
}

// one sweep; with records != NULL the plain method's records of every group
// are logged (the step model is then not applied)
gs2_status sweep_run(gs2_ctx *ctx, gs2_scene *scene, const gs2_camera *cams, int32_t ncam,
                             const float *const *targets, const int32_t *knn, int32_t t, float *records,
                             double *losses_out, int32_t *n_failed, cudaStream_t stream, float *records_damp) {
    TRY(check_scene(ctx, scene));
    REQUIRE(ctx, cams && targets && ncam >= 1 && t >= 0 && t < ncam, GS2_ERR_ARG, "bad cameras or primary index");
    const int K = ctx->cfg.knn_k, f = ctx->cfg.downsample;
    REQUIRE(ctx, K == 0 || knn != nullptr, GS2_ERR_ARG, "knn table is null");
    cudaStream_t st = stream;
    const int nv = 1 + K;
    int vid[17];
    gs2_camera vcam[17];
    const float *vtgt[17];
    vid[0] = t;
    vcam[0] = cams[t];
    vtgt[0] = targets[t];
    TRY(check_cam(ctx, &cams[t]));
    REQUIRE(ctx, targets[t] != nullptr, GS2_ERR_ARG, "null target");
    const size_t slot = 3 * (size_t)(ctx->max_w / f) * (ctx->max_h / f);
    for (int i = 1; i < nv; ++i) {
        const int v = knn[t * K + (i - 1)];
        vid[i] = v;
        if (v < 0) continue;
        REQUIRE(ctx, v < ncam && targets[v] != nullptr, GS2_ERR_ARG, "bad knn entry or null target");
        TRY(check_cam(ctx, &cams[v]));
        gs2_camera_downsample(&cams[v], f, &vcam[i]);
        REQUIRE(ctx, vcam[i].width >= 1 && vcam[i].height >= 1, GS2_ERR_ARG, "secondary too small to downsample");
        float *dst = ctx->sw_tgt + (size_t)(i - 1) * slot;
        if (f > 1) {
            RET_CUDA(ctx, launch_downsample(targets[v], cams[v].width, cams[v].height, f, dst, st));
            vtgt[i] = dst;
        } else {
            vtgt[i] = targets[v];
        }
    }
    if (records) {
        for (int v = 0; v < ncam; ++v) {
            TRY(check_cam(ctx, &cams[v]));
            REQUIRE(ctx, targets[v] != nullptr, GS2_ERR_ARG, "null target");
        }
    }
    const gs2_camera *primary = &cams[t];
    // the views of a group run concurrently: slot 0 on the caller's stream,
    // slot i >= 1 on view lane i - 1 (forked and joined with events); their
    // epilogues add into the shared blocks atomically (the logged sweep keeps
    // one stream: its label passes reuse slot 0's scratch)
    // concurrent views add their epilogues atomically: deterministic mode runs them one after another
    const bool lanes = ctx->view_lanes && !records && nv > 1 && ctx->n_lanes >= nv - 1 && !ctx->cfg.deterministic;
    if (lanes) {
        for (int i = 0; i < nv - 1; ++i) {
            gs2_ctx *l = ctx->lanes[i];
            l->cfg = ctx->cfg;
            l->nb_sort = ctx->nb_sort;
            l->sort_rows = ctx->sort_rows;
            l->accum_px = ctx->accum_px;
            l->accum_split = ctx->accum_split;
        }
    }
    if (ctx->cfg.group_jacobi) {
        // Jacobi over groups: every view rendered once; all groups' blocks from
        // that render; all solves at that state; then the steps applied, the
        // position last (the rotation step turns about the primary's view
        // direction through the unmoved centre)
        REQUIRE(ctx, !records, GS2_ERR_UNSUPPORTED, "the logged sweep runs the groups in series");
        REQUIRE(ctx, ctx->jb_mem != nullptr, GS2_ERR_ARG, "group_jacobi is set but its buffers are missing");
        REQUIRE(ctx, ctx->mlp_w == nullptr && ctx->damp_w == nullptr, GS2_ERR_UNSUPPORTED,
                "the learned networks are trained on the in-series sweep; remove them for group_jacobi");
        const DevScene dsc = make_devscene(scene);
        for (int g = 0; g < 5; ++g)
            RET_CUDA(ctx, cudaMemsetAsync(ctx->jb_blocks[g], 0, blocks_bytes_impl(g, scene->n, scene->sh_degree, nv),
                                          st));
        ctx->stat_slot = ctx->cfg.group_order[0];
        if (lanes) {
            ProjViews pvs;
            pvs.nv = 0;
            for (int i = 0; i < nv; ++i) {
                if (vid[i] < 0) continue;
                gs2_ctx *vc = i > 0 ? ctx->lanes[i - 1] : ctx;
                pvs.cam[pvs.nv] = make_devcam(&vcam[i]);
                pvs.pv[pvs.nv] = proj_view(vc->sw_proj, scene->n);
                if (++pvs.nv == GS2_PROJ_VIEWS) {
                    RET_CUDA(ctx, launch_project_views(dsc, pvs, ctx->cfg, st, ctx->d_status));
                    pvs.nv = 0;
                }
            }
            RET_CUDA(ctx, launch_project_views(dsc, pvs, ctx->cfg, st, ctx->d_status));
            RET_CUDA(ctx, cudaEventRecord(ctx->lane_ev[0], st));
            for (int i = 1; i < nv; ++i) RET_CUDA(ctx, cudaStreamWaitEvent(ctx->lane_st[i - 1], ctx->lane_ev[0], 0));
        }
        for (int i = 0; i < nv; ++i) {
            if (vid[i] < 0) continue;
            gs2_ctx *vc = (lanes && i > 0) ? ctx->lanes[i - 1] : ctx;
            cudaStream_t vs = (lanes && i > 0) ? ctx->lane_st[i - 1] : st;
            gs2_status rc = lanes ? GS2_OK : do_project(vc, scene, &vcam[i], vc->sw_proj, vs);
            if (rc == GS2_OK) rc = do_raster(vc, scene->n, &vcam[i], vc->sw_proj, vc->sw_image, vc->sw_rstate, vs);
            if (rc != GS2_OK) {
                if (vc != ctx) ctx->err = vc->err;
                return rc;
            }
            const int pe = prof_begin(vc, GS2_PROF_LOSS, vs);
            RET_CUDA(ctx, launch_loss(vc->sw_image, vtgt[i], vcam[i].width, vcam[i].height, ctx->cfg, vc->pix_e,
                                      vc->pix_h,
                                      (i == 0 && losses_out) ? losses_out + 2 * ctx->cfg.group_order[0] : nullptr,
                                      vs, ctx->d_status));
            prof_end(vc, pe, vs);
            const ProjView pv = proj_view(vc->sw_proj, scene->n);
            const RasterView rv = raster_view(vc->sw_rstate, vcam[i].width, vcam[i].height);
            for (int gi = 0; gi < 5; ++gi) {
                const int g = ctx->cfg.group_order[gi];
                RET_CUDA(ctx, launch_accum(vc, g, dsc, make_devcam(&vcam[i]), make_devcam(primary), pv, rv, ctx->cfg,
                                           i, ctx->jb_blocks[g], vs));
            }
        }
        if (lanes) {
            for (int i = 1; i < nv; ++i) {
                RET_CUDA(ctx, cudaEventRecord(ctx->lane_ev[i], ctx->lane_st[i - 1]));
                RET_CUDA(ctx, cudaStreamWaitEvent(st, ctx->lane_ev[i], 0));
            }
        }
        for (int gi = 0; gi < 5; ++gi) {
            const int g = ctx->cfg.group_order[gi];
            RET_CUDA(ctx, launch_solve(g, ctx->jb_blocks[g], nv, dsc, make_devcam(primary), ctx->cfg,
                                       ctx->jb_step[g], n_failed, ctx->flags, st, ctx->d_resolves));
        }
        for (int gi = 0; gi < 5; ++gi) {
            const int g = ctx->cfg.group_order[gi];
            if (g != GS2_POS) RET_CUDA(ctx, launch_apply(g, ctx->jb_step[g], dsc, make_devcam(primary), ctx->cfg, st));
        }
        RET_CUDA(ctx, launch_apply(GS2_POS, ctx->jb_step[GS2_POS], dsc, make_devcam(primary), ctx->cfg, st));
        ctx->stat_slot = 0;
        return GS2_OK;
    }
    // the depth order of each view depends on the means and the camera only:
    // the first pass without a valid order sorts and keeps it, later passes
    // reuse it until a position step moves the means
    bool order_valid = false;
    for (int gi = 0; gi < 5; ++gi) {
        const int group = ctx->cfg.group_order[gi];
        ctx->stat_slot = group;
        RET_CUDA(ctx, cudaMemsetAsync(ctx->sw_blocks, 0, blocks_bytes_impl(group, scene->n, scene->sh_degree, nv), st));
        if (lanes) {
            // every view has its own projection buffer here: project them
            // together (the parameters are read once per group, not per view)
            ProjViews pvs;
            pvs.nv = 0;
            for (int i = 0; i < nv; ++i) {
                if (vid[i] < 0) continue;
                gs2_ctx *vc = i > 0 ? ctx->lanes[i - 1] : ctx;
                pvs.cam[pvs.nv] = make_devcam(&vcam[i]);
                pvs.pv[pvs.nv] = proj_view(vc->sw_proj, scene->n);
                if (++pvs.nv == GS2_PROJ_VIEWS) {
                    RET_CUDA(ctx, launch_project_views(make_devscene(scene), pvs, ctx->cfg, st, ctx->d_status));
                    pvs.nv = 0;
                }
            }
            RET_CUDA(ctx, launch_project_views(make_devscene(scene), pvs, ctx->cfg, st, ctx->d_status));
            RET_CUDA(ctx, cudaEventRecord(ctx->lane_ev[0], st));
            for (int i = 1; i < nv; ++i) RET_CUDA(ctx, cudaStreamWaitEvent(ctx->lane_st[i - 1], ctx->lane_ev[0], 0));
        }
        // with a network installed the lanes add into their own blocks (not the
        // colour group, whose views have slots of their own), summed after the join
        const bool own = lanes && (ctx->mlp_w || ctx->damp_w) && group != GS2_COLOR;
        const size_t b1 = blocks_bytes_impl(group, scene->n, scene->sh_degree, 1);
        for (int i = 0; i < nv; ++i) {
            if (vid[i] < 0) continue;
            gs2_ctx *vc = (lanes && i > 0) ? ctx->lanes[i - 1] : ctx;
            cudaStream_t vs = (lanes && i > 0) ? ctx->lane_st[i - 1] : st;
            void *dst = ctx->sw_blocks;
            if (own && i > 0) {
                REQUIRE(ctx, vc->lane_blocks != nullptr, GS2_ERR_ARG, "a view lane has no blocks of its own");
                dst = vc->lane_blocks;
                RET_CUDA(ctx, cudaMemsetAsync(dst, 0, b1, vs));
            }
            // only the position group moves the means: a pass that is not the
            // position pass and finds no valid order sorts each view by depth and
            // keeps the order; the following passes reuse it (the same means and
            // camera give the same order)
            uint32_t *cache = ctx->order_cache + (size_t)i * ctx->max_n;
            gs2_status rc = lanes ? GS2_OK : do_project(vc, scene, &vcam[i], vc->sw_proj, vs);
            if (rc == GS2_OK)
                rc = do_raster(vc, scene->n, &vcam[i], vc->sw_proj, vc->sw_image, vc->sw_rstate, vs,
                               order_valid ? cache : nullptr,
                               (!order_valid && group != GS2_POS) ? cache : nullptr);
            if (rc == GS2_OK)
                rc = do_accum(vc, group, scene, &vcam[i], primary, vc->sw_proj, vc->sw_rstate, vc->sw_image, vtgt[i],
                              i, dst, (i == 0 && losses_out) ? losses_out + 2 * group : nullptr, vs);
            if (rc != GS2_OK) {
                if (vc != ctx) ctx->err = vc->err;
                return rc;
            }
        }
        if (lanes) {
            for (int i = 1; i < nv; ++i) {
                RET_CUDA(ctx, cudaEventRecord(ctx->lane_ev[i], ctx->lane_st[i - 1]));
                RET_CUDA(ctx, cudaStreamWaitEvent(st, ctx->lane_ev[i], 0));
            }
            if (own)
                for (int i = 1; i < nv; ++i)
                    if (vid[i] >= 0)
                        RET_CUDA(ctx, launch_add_floats((float *)ctx->sw_blocks,
                                                        (const float *)ctx->lanes[i - 1]->lane_blocks,
                                                        b1 / sizeof(float), st));
        }
        // a non-position pass stored or reused the views' depth orders; the
        // position step about to be applied invalidates them
        order_valid = group != GS2_POS;
        float *rec = records ? records + (size_t)group * GS2_REC_ROWS * scene->n : nullptr;
        const DevScene dsc = make_devscene(scene);
        if (!rec) {
            TRY(solve_learned(ctx, group, ctx->sw_blocks, nv, scene, primary, ctx->sw_step, n_failed, st));
            RET_CUDA(ctx, launch_apply(group, ctx->sw_step, dsc, make_devcam(primary), ctx->cfg, st));
            continue;
        }
        RET_CUDA(ctx, launch_solve(group, ctx->sw_blocks, nv, dsc, make_devcam(primary), ctx->cfg, ctx->sw_step,
                                   n_failed, ctx->flags, st, ctx->d_resolves));
        // logged: records of the plain step, then the label loss (every view,
        // full resolution) along the step before and after it is applied
        RET_CUDA(ctx, launch_step_records(group, ctx->sw_blocks, nv, dsc, ctx->sw_step, ctx->g_prim, ctx->cfg, rec,
                                          st));
        float *recd = records_damp ? records_damp + (size_t)group * GS2_REC_ROWS * scene->n : nullptr;
        const bool dlab = recd && damping_learned(group) && ctx->cfg.gd_lr[group] <= 0.f;
        if (dlab) {   // the local blocks, kept for the candidate solves; the all-view sum starts at 0
            RET_CUDA(ctx, cudaMemcpyAsync(ctx->lg_bloc, ctx->sw_blocks,
                                          blocks_bytes_impl(group, scene->n, scene->sh_degree, nv),
                                          cudaMemcpyDeviceToDevice, st));
            RET_CUDA(ctx, cudaMemsetAsync(ctx->lg_ball, 0,
                                          blocks_bytes_impl(group, scene->n, scene->sh_degree,
                                                            group == GS2_COLOR ? ncam : 1),
                                          st));
        }
        for (int pass = 0; pass < 2; ++pass) {
            float *phi = pass == 0 ? rec + (size_t)GS2_MLP_NFEAT * scene->n : ctx->lg_phi;
            RET_CUDA(ctx, cudaMemsetAsync(phi, 0, sizeof(float) * scene->n, st));
            for (int v = 0; v < ncam; ++v) {
                RET_CUDA(ctx, cudaMemsetAsync(ctx->sw_blocks, 0, b1, st));
                TRY(do_project(ctx, scene, &cams[v], ctx->sw_proj, st));
                TRY(do_raster(ctx, scene->n, &cams[v], ctx->sw_proj, ctx->sw_image, ctx->sw_rstate, st));
                TRY(do_accum(ctx, group, scene, &cams[v], primary, ctx->sw_proj, ctx->sw_rstate, ctx->sw_image,
                             targets[v], 0, ctx->sw_blocks, nullptr, st, false));
                RET_CUDA(ctx, launch_phi_add(group, ctx->sw_blocks, dsc, ctx->sw_step, phi, st));
                if (pass == 0 && dlab) {   // sum of the views' blocks (colour: view v in slot v)
                    if (group == GS2_COLOR)
                        RET_CUDA(ctx, cudaMemcpyAsync((char *)ctx->lg_ball + (size_t)v * b1, ctx->sw_blocks, b1,
                                                      cudaMemcpyDeviceToDevice, st));
                    else
                        RET_CUDA(ctx, launch_add_floats((float *)ctx->lg_ball, (const float *)ctx->sw_blocks,
                                                        b1 / sizeof(float), st));
                }
            }
            if (pass == 0 && recd) {   // damping labels: candidate steps of the same solve, scored on the all-view model
                if (dlab) {
                    gs2_config cj = ctx->cfg;
                    for (int j = 0; j < 7; ++j) {   // rho = 10^0, 10^0.5, .., 10^3
                        const float rj = exp10f(0.5f * (float)j);
                        cj.damping_mu0 = ctx->cfg.damping_mu0 * rj;
                        RET_CUDA(ctx, launch_solve(group, ctx->lg_bloc, nv, dsc, make_devcam(primary), cj,
                                                   ctx->lg_step2, nullptr, ctx->flags, st, nullptr));
                        RET_CUDA(ctx, launch_damp_eval(group, ctx->lg_ball, group == GS2_COLOR ? ncam : 1, dsc,
                                                       ctx->lg_step2, ctx->cfg, rj, ctx->lg_bq, ctx->lg_brho,
                                                       ctx->lg_wq, j == 0, st));
                    }
                }
                RET_CUDA(ctx, launch_damp_labels(group, rec, dlab ? ctx->lg_bq : nullptr, ctx->lg_wq, ctx->lg_brho,
                                                 scene->n, recd, st));
            }
            if (pass == 0)
                RET_CUDA(ctx, launch_apply(group, ctx->sw_step, dsc, make_devcam(primary), ctx->cfg, st));
        }
        RET_CUDA(ctx, launch_step_labels(group, nullptr, 1, dsc, ctx->sw_step, ctx->lg_phi, rec, st));
    }
    ctx->stat_slot = 0;
    return GS2_OK;
}

extern "C" gs2_status gs2_sweep(gs2_ctx *ctx, gs2_scene *scene, const gs2_camera *cams, int32_t ncam,
                                const float *const *targets, const int32_t *knn, int32_t t, double *losses_out,
                                int32_t *n_failed, gs2_stream stream) {
    if (!ctx) return GS2_ERR_ARG;
    return sweep_run(ctx, scene, cams, ncam, targets, knn, t, nullptr, losses_out, n_failed, (cudaStream_t)stream);
}

extern "C" gs2_status gs2_sweep_logged(gs2_ctx *ctx, gs2_scene *scene, const gs2_camera *cams, int32_t ncam,
                                       const float *const *targets, const int32_t *knn, int32_t t, float *records,
                                       float *records_damping, double *losses_out, int32_t *n_failed,
                                       gs2_stream stream) {
    if (!ctx) return GS2_ERR_ARG;
    REQUIRE(ctx, records != nullptr, GS2_ERR_ARG, "records is null");
    if (records_damping) {   // scratch of the damping labels, sized for this scene and camera count
        TRY(check_scene(ctx, scene));
        REQUIRE(ctx, ncam >= 1, GS2_ERR_ARG, "bad camera count");
        const int n = scene->n, sh = scene->sh_degree, nv = 1 + ctx->cfg.knn_k;
        size_t ball = 0, bloc = 0;
        for (int g = 0; g < 5; ++g) {
            ball = std::max(ball, blocks_bytes_impl(g, n, sh, g == GS2_COLOR ? ncam : 1));
            bloc = std::max(bloc, blocks_bytes_impl(g, n, sh, nv));
        }
        if (ball > ctx->lg_ball_bytes || bloc > ctx->lg_bloc_bytes || !ctx->lg_bq) {
            RET_CUDA(ctx, cudaDeviceSynchronize());
            void *ptrs[] = {ctx->lg_ball, ctx->lg_bloc, ctx->lg_step2, ctx->lg_bq, ctx->lg_brho, ctx->lg_wq};
            for (void *p : ptrs)
                if (p) cudaFree(p);
            ctx->lg_ball = ctx->lg_bloc = ctx->lg_step2 = nullptr;
            ctx->lg_bq = ctx->lg_brho = ctx->lg_wq = nullptr;
            ctx->lg_ball_bytes = ctx->lg_bloc_bytes = 0;
            RET_CUDA(ctx, cudaMalloc(&ctx->lg_ball, ball));
            RET_CUDA(ctx, cudaMalloc(&ctx->lg_bloc, bloc));
            RET_CUDA(ctx, cudaMalloc(&ctx->lg_step2, ctx->sw_step_bytes));
            RET_CUDA(ctx, cudaMalloc((void **)&ctx->lg_bq, sizeof(float) * (size_t)ctx->max_n));
            RET_CUDA(ctx, cudaMalloc((void **)&ctx->lg_brho, sizeof(float) * (size_t)ctx->max_n));
            RET_CUDA(ctx, cudaMalloc((void **)&ctx->lg_wq, sizeof(float) * (size_t)ctx->max_n));
            ctx->lg_ball_bytes = ball;
            ctx->lg_bloc_bytes = bloc;
        }
    }
    return sweep_run(ctx, scene, cams, ncam, targets, knn, t, records, losses_out, n_failed, (cudaStream_t)stream,
                     records_damping);
}

extern "C" uint64_t gs2_launch_count(void) { return g_gs2_launches.load(); }

extern "C" gs2_status gs2_profile(gs2_ctx *ctx, int32_t enable) {
    if (!ctx) return GS2_ERR_ARG;
    if (enable && !ctx->prof_ev[0])
        for (int i = 0; i < 2 * GS2_PROF_POOL; ++i) RET_CUDA(ctx, cudaEventCreate(&ctx->prof_ev[i]));
    RET_CUDA(ctx, cudaDeviceSynchronize());
    ctx->prof_on = enable ? 1 : 0;
    ctx->prof_n = 0;
    ctx->stat_slot = 0;
    for (int g = 0; g < 5; ++g) ctx->h_pixels[g] = 0;
    RET_CUDA(ctx, cudaMemset(ctx->d_stats, 0, sizeof(unsigned long long) * 25));
    return GS2_OK;
}

extern "C" gs2_status gs2_profile_read(gs2_ctx *ctx, double *accum_ms, int64_t *accum_launches, uint64_t *stats) {
    if (!ctx || !accum_ms || !accum_launches || !stats) return GS2_ERR_ARG;
    RET_CUDA(ctx, cudaDeviceSynchronize());
    for (int g = 0; g < 5; ++g) {
        accum_ms[g] = 0.0;
        accum_launches[g] = 0;
    }
    for (int i = 0; i < ctx->prof_n; ++i) {
        if (ctx->prof_group[i] >= 5) continue;   // a stage, not an accumulation
        float ms = 0.f;
        RET_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->prof_ev[2 * i], ctx->prof_ev[2 * i + 1]));
        accum_ms[ctx->prof_group[i]] += ms;
        accum_launches[ctx->prof_group[i]] += 1;
    }
    unsigned long long h[25];
    RET_CUDA(ctx, cudaMemcpy(h, ctx->d_stats, sizeof(h), cudaMemcpyDeviceToHost));
    for (int g = 0; g < 5; ++g) {
        stats[6 * g + 0] = h[5 * g + 0];
        stats[6 * g + 1] = h[5 * g + 1];
        stats[6 * g + 2] = h[5 * g + 2];
        stats[6 * g + 3] = ctx->h_pixels[g];
        stats[6 * g + 4] = h[5 * g + 3];
        stats[6 * g + 5] = h[5 * g + 4];
    }
    return GS2_OK;
}

extern "C" gs2_status gs2_profile_read_stages(gs2_ctx *ctx, double *ms_out, int64_t *count_out) {
    if (!ctx || !ms_out || !count_out) return GS2_ERR_ARG;
    RET_CUDA(ctx, cudaDeviceSynchronize());
    for (int k = 0; k < 3; ++k) {
        ms_out[k] = 0.0;
        count_out[k] = 0;
    }
    for (int i = 0; i < ctx->prof_n; ++i) {
        const int k = ctx->prof_group[i] - GS2_PROF_BIN;
        if (k < 0 || k > 2) continue;
        float ms = 0.f;
        RET_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->prof_ev[2 * i], ctx->prof_ev[2 * i + 1]));
        ms_out[k] += ms;
        count_out[k] += 1;
    }
    return GS2_OK;
}

int prof_begin(gs2_ctx *ctx, int tag, cudaStream_t st) {
    gs2_ctx *pc = ctx->owner ? ctx->owner : ctx;
    if (!pc->prof_on || pc->prof_n >= GS2_PROF_POOL) return -1;
    const int i = pc->prof_n++;
    pc->prof_group[i] = tag;
    cudaEventRecord(pc->prof_ev[2 * i], st);
    return i;
}

void prof_end(gs2_ctx *ctx, int idx, cudaStream_t st) {
    if (idx < 0) return;
    gs2_ctx *pc = ctx->owner ? ctx->owner : ctx;
    cudaEventRecord(pc->prof_ev[2 * idx + 1], st);
}

extern "C" gs2_status gs2_fp64_resolves(gs2_ctx *ctx, uint64_t *out, int32_t reset) {
    if (!ctx || !out) return GS2_ERR_ARG;
    unsigned long long h[5];
    RET_CUDA(ctx, cudaDeviceSynchronize());
    RET_CUDA(ctx, cudaMemcpy(h, ctx->d_resolves, sizeof(h), cudaMemcpyDeviceToHost));
    for (int g = 0; g < 5; ++g) out[g] = h[g];
    if (reset) RET_CUDA(ctx, cudaMemset(ctx->d_resolves, 0, sizeof(h)));
    return GS2_OK;
}

// ------------------------------------------------------------------ introspection
__global__ void k_unpack_proj(ProjView pv, int n, float *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float4 a = pv.recA[k], b = pv.recB[k], c = pv.col[k];
    const uint2 r = pv.rect[k];
    const float v[GS2_DEBUG_PROJ_ROWS] = {a.x, a.y, a.z, a.w, b.x, b.y, c.x, c.y, c.z, __uint_as_float(pv.key[k]),
                                          (float)pv.touched[k], b.z, b.w, pv.k2[k], c.w, __uint_as_float(r.x),
                                          __uint_as_float(r.y), 0.f};
    for (int i = 0; i < GS2_DEBUG_PROJ_ROWS; ++i) out[(size_t)i * n + k] = v[i];
}

extern "C" gs2_status gs2_debug_proj(const void *proj, int64_t n, float *out, gs2_stream stream) {
    if (!proj || !out || n < 0) return GS2_ERR_ARG;
    if (n == 0) return GS2_OK;
    k_unpack_proj<<<(int)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(proj_view(const_cast<void *>(proj), n),
                                                                            (int)n, out);
    return cudaGetLastError() == cudaSuccess ? GS2_OK : GS2_ERR_CUDA;
}

extern "C" gs2_status gs2_debug_lookback_timeout(gs2_ctx *ctx, int32_t chunk, uint32_t limit, gs2_stream stream) {
    if (!ctx || chunk < 1 || chunk >= GS2_SCAN_CHUNKS || limit < 1 || limit > (1u << 20)) return GS2_ERR_ARG;
    RET_CUDA(ctx, launch_debug_lookback(ctx, chunk, limit, (cudaStream_t)stream));
    return GS2_OK;
}

extern "C" gs2_status gs2_debug_keys(const void *proj, int64_t n, uint32_t *keys_out, gs2_stream stream) {
    if (!proj || !keys_out || n < 0) return GS2_ERR_ARG;
    ProjView pv = proj_view(const_cast<void *>(proj), n);
    return cudaMemcpyAsync(keys_out, pv.key, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice,
                           (cudaStream_t)stream) == cudaSuccess
               ? GS2_OK
               : GS2_ERR_CUDA;
}

extern "C" gs2_status gs2_debug_tiles(gs2_ctx *ctx, uint32_t *ranges_out, uint32_t *ids_out, int64_t capacity,
                                      int64_t *n_pairs_out, gs2_stream stream) {
    if (!ctx || !ranges_out || !ids_out || !n_pairs_out) return GS2_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t cnt[4];
    RET_CUDA(ctx, cudaMemcpyAsync(cnt, ctx->d_count, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    RET_CUDA(ctx, cudaStreamSynchronize(st));
    *n_pairs_out = cnt[3];   // the listed pairs
    const size_t ntiles = (size_t)ctx->tiles_x * ctx->tiles_y;
    RET_CUDA(ctx, cudaMemcpyAsync(ranges_out, ctx->ranges, sizeof(uint2) * ntiles, cudaMemcpyDeviceToDevice, st));
    const size_t m = std::min<size_t>(cnt[3], (size_t)std::max<int64_t>(capacity, 0));
    if (m) RET_CUDA(ctx, cudaMemcpyAsync(ids_out, ctx->list_ids, sizeof(uint32_t) * m,
                                         cudaMemcpyDeviceToDevice, st));
    return GS2_OK;
}
