// Batched sweeps over many independent scenes, kernel tuning and its autotuner
// (an extension for throughput over many scenes; the paper trains one scene).
//
// gs2_batch owns one context and one stream per scene.  A batched sweep forks
// every scene's sweep (Sec. 4.2 groups with the Sec. 4.3 secondaries) onto its
// stream from the caller's stream and joins them back, so scenes of uneven
// size fill the 148 SMs together: small scenes' kernels run beside a large
// scene's instead of after it.
//
// use_graph = 1: the whole fork/join is captured as one CUDA graph (one
// parallel branch per scene) and launched with a single cudaGraphLaunch;
// later calls re-capture (the primaries change from sweep to sweep, and with
// them the kernels' camera arguments) and update the instantiated graph in
// place with cudaGraphExecUpdate (accepted while the kernel sequence is the
// same).
// use_graph = 2: one graph per scene and sweep inputs, kept: the inputs that
// end up in kernel arguments (primary, the cameras of its views, target,
// scene and output pointers, configuration, step model, tuning) are hashed;
// a sweep whose key was seen before replays its instantiated graph without
// any capture -- in training the primaries cycle through the cameras, so
// every graph is captured once and replayed from then on.
//
// Tuning: the radix sort's grid (CTAs) and keys per thread per scatter round.
// The autotuner times whole sweeps on a scratch copy of the scene for every
// candidate and keeps the fastest in the context.
#include <string>
#include <unordered_map>
#include <vector>

#include "common.cuh"

#define RETC(expr)                                  \
    do {                                            \
        if ((expr) != cudaSuccess) return GS2_ERR_CUDA; \
    } while (0)

// batch variant: records the failing call in the batch
#define RETB(b, expr)                                                                  \
    do {                                                                               \
        const cudaError_t e_ = (expr);                                                 \
        if (e_ != cudaSuccess) {                                                       \
            (b)->err = std::string(#expr) + ": " + cudaGetErrorString(e_);             \
            return GS2_ERR_CUDA;                                                       \
        }                                                                              \
    } while (0)

extern "C" gs2_status gs2_get_tuning(const gs2_ctx *ctx, gs2_tuning *out) {
    if (!ctx || !out) return GS2_ERR_ARG;
    out->sort_blocks = ctx->nb_sort;
    out->sort_rows = ctx->sort_rows;
    out->view_lanes = ctx->view_lanes;
    out->accum_px = ctx->accum_px;
    out->accum_split = ctx->accum_split;
    return GS2_OK;
}

extern "C" gs2_status gs2_set_tuning(gs2_ctx *ctx, const gs2_tuning *t) {
    if (!ctx || !t) return GS2_ERR_ARG;
    if (t->sort_blocks < 1 || t->sort_blocks > GS2_SORT_BLOCKS_MAX) return GS2_ERR_ARG;
    if (t->sort_rows != 2 && t->sort_rows != 4 && t->sort_rows != 8 && t->sort_rows != 16) return GS2_ERR_ARG;
    if (t->view_lanes != 0 && t->view_lanes != 1) return GS2_ERR_ARG;
    if (t->accum_px != 2 && !(t->accum_px == 4 && GS2_TILE == 16)) return GS2_ERR_ARG;
    if (t->accum_split < 0 || t->accum_split > GS2_SPLIT_MAX || t->accum_split % GS2_TILE_PIX != 0)
        return GS2_ERR_ARG;
    if (!ensure_split(ctx, t->accum_split)) return GS2_ERR_OOM;
    ctx->nb_sort = t->sort_blocks;
    ctx->sort_rows = t->sort_rows;
    ctx->view_lanes = t->view_lanes;
    ctx->accum_px = t->accum_px;
    ctx->accum_split = t->accum_split;
    return GS2_OK;
}

extern "C" gs2_status gs2_autotune(gs2_ctx *ctx, const gs2_scene *scene, const gs2_camera *cams, int32_t ncam,
                                   const float *const *targets, const int32_t *knn, int32_t t, int32_t reps,
                                   gs2_tuning *best_out, float *best_ms_out, gs2_stream stream) {
    if (!ctx || !scene || !cams || !targets || reps < 1 || ncam < 1 || t < 0 || t >= ncam) return GS2_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int n = scene->n, S = sh_count(scene->sh_degree);
    // scratch copy of the scene: the timed sweeps must not move the caller's
    const size_t floats = (size_t)n * (3 + 4 + 3 + 1 + 3 * (size_t)S);
    float *buf = nullptr;
    if (cudaMalloc(&buf, sizeof(float) * (floats > 0 ? floats : 1)) != cudaSuccess) return GS2_ERR_OOM;
    gs2_scene cp = *scene;
    cp.mean = buf;
    cp.quat = cp.mean + 3 * (size_t)n;
    cp.scale = cp.quat + 4 * (size_t)n;
    cp.opacity = cp.scale + 3 * (size_t)n;
    cp.sh = cp.opacity + (size_t)n;
    auto reset = [&]() {
        return cudaMemcpyAsync(cp.mean, scene->mean, sizeof(float) * 3 * n, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
               cudaMemcpyAsync(cp.quat, scene->quat, sizeof(float) * 4 * n, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
               cudaMemcpyAsync(cp.scale, scene->scale, sizeof(float) * 3 * n, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
               cudaMemcpyAsync(cp.opacity, scene->opacity, sizeof(float) * n, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
               cudaMemcpyAsync(cp.sh, scene->sh, sizeof(float) * 3 * S * (size_t)n, cudaMemcpyDeviceToDevice, st) ==
                   cudaSuccess;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gs2_status rc = GS2_OK;
    const gs2_tuning keep = {ctx->nb_sort, ctx->sort_rows, ctx->view_lanes, ctx->accum_px, ctx->accum_split};
    gs2_tuning best = keep;
    float best_ms = 1e30f;
    const int blocks[3] = {148 * 2, 148 * 4, 148 * 6};
    const int rows[4] = {2, 4, 8, 16};
    // ms per sweep of one candidate (one untimed sweep for first-touch effects, then `reps` timed)
    auto trial = [&](const gs2_tuning &c) {
        ctx->nb_sort = c.sort_blocks;
        ctx->sort_rows = c.sort_rows;
        ctx->accum_px = c.accum_px;
        ctx->accum_split = c.accum_split;
        if (!reset()) { rc = GS2_ERR_CUDA; return; }
        rc = sweep_run(ctx, &cp, cams, ncam, targets, knn, t, nullptr, nullptr, nullptr, st);
        if (rc != GS2_OK) return;
        if (!reset() || cudaEventRecord(e0, st) != cudaSuccess) { rc = GS2_ERR_CUDA; return; }
        for (int r = 0; r < reps && rc == GS2_OK; ++r)
            rc = sweep_run(ctx, &cp, cams, ncam, targets, knn, t, nullptr, nullptr, nullptr, st);
        if (rc != GS2_OK) return;
        float ms = 0.f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { rc = GS2_ERR_CUDA; return; }
        ms /= (float)reps;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = GS2_ERR_CUDA;
    // the sort grid first (at the current accumulation shape), then the
    // accumulation's pixels per thread at the best sort setting
    for (int bi = 0; bi < 3 && rc == GS2_OK; ++bi)
        for (int ri = 0; ri < 4 && rc == GS2_OK; ++ri)
            trial({blocks[bi], rows[ri], ctx->view_lanes, keep.accum_px, keep.accum_split});
    const int pxs[2] = {2, 4};
    for (int pi = 0; pi < (GS2_TILE == 16 ? 2 : 1) && rc == GS2_OK; ++pi)
        if (pxs[pi] != keep.accum_px)
            trial({best.sort_blocks, best.sort_rows, best.view_lanes, pxs[pi], keep.accum_split});
    // then the split walks (off, and chunks of 1 and 4 compositing batches)
    const int splits[3] = {0, GS2_TILE_PIX, 4 * GS2_TILE_PIX};
    if (rc == GS2_OK && !ensure_split(ctx, GS2_TILE_PIX)) rc = GS2_ERR_OOM;
    for (int si = 0; si < 3 && rc == GS2_OK; ++si)
        if (splits[si] != keep.accum_split)
            trial({best.sort_blocks, best.sort_rows, best.view_lanes, best.accum_px, splits[si]});
    cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (rc != GS2_OK) {
        ctx->nb_sort = keep.sort_blocks;
        ctx->sort_rows = keep.sort_rows;
        ctx->accum_px = keep.accum_px;
        ctx->accum_split = keep.accum_split;
        return rc;
    }
    ctx->nb_sort = best.sort_blocks;
    ctx->sort_rows = best.sort_rows;
    ctx->accum_px = best.accum_px;
    ctx->accum_split = best.accum_split;
    if (best_out) *best_out = best;
    if (best_ms_out) *best_ms_out = best_ms;
    return GS2_OK;
}

// ------------------------------------------------------------------ batch
#define GS2_GRAPH_CACHE_MAX 512   // per scene; beyond it the cache is emptied and refilled

struct gs2_batch {
    std::vector<gs2_ctx *> ctx;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr, ready = nullptr;
    cudaStream_t cap = nullptr;   // capture origin (the caller's stream may be the legacy default stream)
    cudaGraphExec_t exec = nullptr;
    int graph_updates = 0, graph_instantiations = 0, graph_replays = 0;
    std::vector<std::unordered_map<uint64_t, cudaGraphExec_t>> cache;   // per scene (use_graph = 2)
    std::string err;
};

// FNV-1a over raw bytes
static inline void fnv(uint64_t &h, const void *p, size_t nbytes) {
    const unsigned char *c = (const unsigned char *)p;
    for (size_t i = 0; i < nbytes; ++i) {
        h ^= c[i];
        h *= 1099511628211ull;
    }
}

static void batch_free(gs2_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto &m : b->cache)
        for (auto &kv : m) cudaGraphExecDestroy(kv.second);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->ready) cudaEventDestroy(b->ready);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamDestroy(s);
    for (gs2_ctx *c : b->ctx)
        if (c) gs2_destroy(c);
}

extern "C" gs2_status gs2_batch_create(gs2_batch **out, const gs2_config *cfg, int32_t n_scenes,
                                       const gs2_batch_scene *desc) {
    if (!out || n_scenes < 1 || !desc) return GS2_ERR_ARG;
    *out = nullptr;
    gs2_batch *b = new (std::nothrow) gs2_batch();
    if (!b) return GS2_ERR_OOM;
    b->ctx.assign(n_scenes, nullptr);
    b->streams.assign(n_scenes, nullptr);
    b->join.assign(n_scenes, nullptr);
    b->cache.resize(n_scenes);
    gs2_status rc = GS2_OK;
    for (int i = 0; i < n_scenes && rc == GS2_OK; ++i) {
        rc = gs2_create(&b->ctx[i], cfg, desc[i].max_gaussians, desc[i].max_width, desc[i].max_height,
                        desc[i].max_sh_degree, desc[i].max_pairs);
        if (rc == GS2_OK && (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
                             cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) != cudaSuccess))
            rc = GS2_ERR_CUDA;
    }
    if (rc == GS2_OK && (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming) != cudaSuccess ||
                         cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess))
        rc = GS2_ERR_CUDA;
    if (rc != GS2_OK) {
        batch_free(b);
        delete b;
        cudaGetLastError();
        return rc;
    }
    *out = b;
    return GS2_OK;
}

extern "C" gs2_status gs2_batch_destroy(gs2_batch *b) {
    if (!b) return GS2_ERR_ARG;
    batch_free(b);
    delete b;
    return GS2_OK;
}

extern "C" gs2_ctx *gs2_batch_ctx(gs2_batch *b, int32_t i) {
    if (!b || i < 0 || i >= (int)b->ctx.size()) return nullptr;
    return b->ctx[i];
}

extern "C" const char *gs2_batch_last_error(const gs2_batch *b) { return b ? b->err.c_str() : "null batch"; }

extern "C" gs2_status gs2_batch_stats(const gs2_batch *b, int32_t *instantiations, int32_t *updates,
                                      int32_t *replays) {
    if (!b) return GS2_ERR_ARG;
    if (instantiations) *instantiations = b->graph_instantiations;
    if (updates) *updates = b->graph_updates;
    if (replays) *replays = b->graph_replays;
    return GS2_OK;
}

// key of everything a scene's sweep bakes into kernel arguments
static uint64_t sweep_key(const gs2_ctx *c, const gs2_scene *scene, const gs2_camera *cams, int32_t ncam,
                          const float *const *targets, const int32_t *knn, int32_t t, const double *losses,
                          const int32_t *n_failed) {
    uint64_t h = 1469598103934665603ull;
    fnv(h, scene, sizeof(*scene));
    fnv(h, &t, sizeof(t));
    fnv(h, &ncam, sizeof(ncam));
    fnv(h, &cams[t], sizeof(gs2_camera));
    fnv(h, &targets[t], sizeof(targets[t]));
    const int K = c->cfg.knn_k;
    for (int q = 0; q < K; ++q) {
        const int v = knn[t * K + q];
        fnv(h, &v, sizeof(v));
        if (v >= 0 && v < ncam) {
            fnv(h, &cams[v], sizeof(gs2_camera));
            fnv(h, &targets[v], sizeof(targets[v]));
        }
    }
    fnv(h, &losses, sizeof(losses));
    fnv(h, &n_failed, sizeof(n_failed));
    fnv(h, &c->cfg, sizeof(c->cfg));
    fnv(h, &c->mlp_w, sizeof(c->mlp_w));
    fnv(h, &c->damp_w, sizeof(c->damp_w));
    fnv(h, &c->nb_sort, sizeof(c->nb_sort));
    fnv(h, &c->sort_rows, sizeof(c->sort_rows));
    fnv(h, &c->view_lanes, sizeof(c->view_lanes));
    fnv(h, &c->accum_px, sizeof(c->accum_px));
    fnv(h, &c->accum_split, sizeof(c->accum_split));
    // buffers that a tuning change can reallocate (the split walks'
    // checkpoints and items, of the context and its view lanes): a graph
    // captured with the old ones must not match
    for (int i = -1; i < c->n_lanes; ++i) {
        const gs2_ctx *l = i < 0 ? c : c->lanes[i];
        if (!l) continue;
        fnv(h, &l->ck, sizeof(l->ck));
        fnv(h, &l->tile_maxlast, sizeof(l->tile_maxlast));
        fnv(h, &l->acc_items, sizeof(l->acc_items));
        fnv(h, &l->acc_ctrl, sizeof(l->acc_ctrl));
    }
    return h;
}

// use_graph = 2: per scene, replay the graph of this sweep's key or capture it
static gs2_status batch_cached(gs2_batch *b, gs2_scene *scenes, const gs2_camera *const *cams, const int32_t *ncam,
                               const float *const *const *targets, const int32_t *const *knn, const int32_t *t,
                               double *losses, int32_t *n_failed, cudaStream_t st) {
    const int ns = (int)b->ctx.size();
    RETB(b, cudaEventRecord(b->fork, st));
    for (int i = 0; i < ns; ++i) {
        double *li = losses ? losses + 10 * (size_t)i : nullptr;
        int32_t *fi = n_failed ? n_failed + i : nullptr;
        const uint64_t key = sweep_key(b->ctx[i], &scenes[i], cams[i], ncam[i], targets[i], knn[i], t[i], li, fi);
        auto &m = b->cache[i];
        auto it = m.find(key);
        cudaGraphExec_t exec = nullptr;
        if (it != m.end()) {
            exec = it->second;
            ++b->graph_replays;
        } else {
            if ((int)m.size() >= GS2_GRAPH_CACHE_MAX) {
                for (auto &kv : m) cudaGraphExecDestroy(kv.second);
                m.clear();
            }
            RETB(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
            const gs2_status rc = sweep_run(b->ctx[i], &scenes[i], cams[i], ncam[i], targets[i], knn[i], t[i], nullptr,
                                            li, fi, b->cap);
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(b->cap, &g);
            if (rc != GS2_OK) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                b->err = "scene " + std::to_string(i) + ": " + b->ctx[i]->err;
                return rc;
            }
            if (ec != cudaSuccess || !g) {
                b->err = std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ec);
                return GS2_ERR_CUDA;
            }
            const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) {
                b->err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei);
                return GS2_ERR_CUDA;
            }
            m.emplace(key, exec);
            ++b->graph_instantiations;
        }
        RETB(b, cudaStreamWaitEvent(b->streams[i], b->fork, 0));
        RETB(b, cudaGraphLaunch(exec, b->streams[i]));
        RETB(b, cudaEventRecord(b->join[i], b->streams[i]));
        RETB(b, cudaStreamWaitEvent(st, b->join[i], 0));
    }
    return GS2_OK;
}

// fork, every scene's sweep on its stream, join
static gs2_status batch_enqueue(gs2_batch *b, gs2_scene *scenes, const gs2_camera *const *cams,
                                const int32_t *ncam, const float *const *const *targets,
                                const int32_t *const *knn, const int32_t *t, double *losses, int32_t *n_failed,
                                cudaStream_t st) {
    const int ns = (int)b->ctx.size();
    RETB(b, cudaEventRecord(b->fork, st));
    for (int i = 0; i < ns; ++i) {
        RETB(b, cudaStreamWaitEvent(b->streams[i], b->fork, 0));
        const gs2_status rc = sweep_run(b->ctx[i], &scenes[i], cams[i], ncam[i], targets[i], knn[i], t[i], nullptr,
                                        losses ? losses + 10 * (size_t)i : nullptr, n_failed ? n_failed + i : nullptr,
                                        b->streams[i]);
        if (rc != GS2_OK) {
            b->err = "scene " + std::to_string(i) + ": " + b->ctx[i]->err;
            return rc;
        }
        RETB(b, cudaEventRecord(b->join[i], b->streams[i]));
        RETB(b, cudaStreamWaitEvent(st, b->join[i], 0));
    }
    return GS2_OK;
}

extern "C" gs2_status gs2_batch_sweep(gs2_batch *b, gs2_scene *scenes, const gs2_camera *const *cams,
                                      const int32_t *ncam, const float *const *const *targets,
                                      const int32_t *const *knn, const int32_t *t, double *losses_out,
                                      int32_t *n_failed, int32_t use_graph, gs2_stream stream) {
    if (!b || !scenes || !cams || !ncam || !targets || !knn || !t) return GS2_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (!use_graph) return batch_enqueue(b, scenes, cams, ncam, targets, knn, t, losses_out, n_failed, st);
    if (use_graph == 2) return batch_cached(b, scenes, cams, ncam, targets, knn, t, losses_out, n_failed, st);
    // capture on the batch's own stream; the graph is launched on the caller's
    RETB(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    const gs2_status rc = batch_enqueue(b, scenes, cams, ncam, targets, knn, t, losses_out, n_failed, b->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->cap, &g);   // always ends the capture
    if (rc != GS2_OK) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc;
    }
    if (ec != cudaSuccess || !g) {
        b->err = std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ec);
        return GS2_ERR_CUDA;
    }
    bool ready = false;
    if (b->exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(b->exec, g, &info) == cudaSuccess) {
            ready = true;
            ++b->graph_updates;
        } else {
            cudaGetLastError();
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
    }
    if (!ready) {
        const cudaError_t ei = cudaGraphInstantiate(&b->exec, g, 0);
        if (ei != cudaSuccess) {
            cudaGraphDestroy(g);
            b->exec = nullptr;
            b->err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei);
            return GS2_ERR_CUDA;
        }
        ++b->graph_instantiations;
    }
    cudaGraphDestroy(g);
    RETB(b, cudaGraphLaunch(b->exec, st));
    return GS2_OK;
}
