// gs2_raster_fwd compositing (Eq. 3dgs): one CTA per screen tile (16x16), one
// thread per pixel, the tile's depth-sorted Gaussian list staged through
// shared memory in batches of 256 records (one record gather per thread per
// batch, copied asynchronously into the second buffer while the first is
// walked; the per-pixel inner loop reads shared memory only).
//   alpha = min(sigma G, alpha_max); skip alpha < alpha_min; stop before
//   T (1 - alpha) < t_min; c += alpha T c~; black background.  Whether a term
//   is skipped or clamped is decided from its quadratic form q against the
//   Gaussian's thresholds l, lmax (decide.cuh), reproducibly.
// Writes the planar image, the final transmittance and the list position
// after the last contributor (consumed by the accumulation pass).
// CK (the split accumulation's checkpoints, rv.ck): at every multiple c_j of
// rv.ck_every list entries the tile's walk reaches, each pixel's T(c_j) and
// the colour its entries from c_j on add (sum of alpha T c~, kept per segment
// between checkpoints and summed from the back once the walk ends: no
// difference of two nearly equal colours, which would lose the digits of a
// deep T; the pixel's colour is then the sum of its segments, added back to
// front), and the tile's walk length (the largest list position after a last
// contributor).
#include "common.cuh"

template <bool CK>
__global__ void __launch_bounds__(GS2_TILE_PIX) k_raster(const uint2 *__restrict__ ranges,
                                                         const uint32_t *__restrict__ ids, ProjView pv, int W, int H,
                                                         int tiles_x, float amin, float amax, float tmin,
                                                         float *__restrict__ image, RasterView rv,
                                                         const uint32_t *__restrict__ tile_order) {
    // two staging buffers: batch b + 1 is copied in (cp.async) while batch b is walked
    __shared__ float4 sA[2][GS2_TILE_PIX], sB[2][GS2_TILE_PIX], sC[2][GS2_TILE_PIX];
    __shared__ uint32_t sMax;
    const int t = threadIdx.x;
    const int tile = tile_order ? (int)tile_order[blockIdx.x] : (int)blockIdx.x;   // longest lists first
    const int tcol = tile % tiles_x, trow = tile / tiles_x;
    const int px = tcol * GS2_TILE + gs2_tile_px(t), py = trow * GS2_TILE + gs2_tile_py(t);
    const bool inside = px < W && py < H;
    bool done = !inside;
    const uint2 r = ranges[tile];
    const int n = (int)(r.y - r.x);
    const float fx = (float)px, fy = (float)py;
    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;   // CK: colour of the current segment
    uint32_t lastc = 0u;
    const int nbat = (n + GS2_TILE_PIX - 1) / GS2_TILE_PIX;
    // checkpoint j (list position j ck_every, j >= 1) of this tile goes to slot
    // r.x / ck_every + j: distinct for all tiles, below (list length) / ck_every
    const int ck_b = CK ? rv.ck_every / GS2_TILE_PIX : 1;   // batches between checkpoints
    const size_t ck_base = CK ? (size_t)(r.x / (uint32_t)rv.ck_every) : 0;
    const int lp = gs2_tile_py(t) * GS2_TILE + gs2_tile_px(t);   // row-major pixel of the tile
    int nck = 0;   // checkpoints written (CTA-uniform)
    auto issue = [&](int b, uint32_t k) {
        const int buf = b & 1;
        if (b * GS2_TILE_PIX + t < n) {
            cp_async16(&sA[buf][t], &pv.recA[k]);
            cp_async16(&sB[buf][t], &pv.recB[k]);
            cp_async16(&sC[buf][t], &pv.col[k]);
        }
        cp_async_commit();
    };
    uint32_t knext = 0u;
    if (nbat > 0) {
        if (t < n) knext = ids[r.x + t];
        issue(0, knext);
        if (GS2_TILE_PIX + t < n) knext = ids[r.x + GS2_TILE_PIX + t];
    }
    for (int b = 0; b < nbat; ++b) {
        cp_async_wait_all();
        if (__syncthreads_count(done) == GS2_TILE_PIX) break;   // also: batch b visible, b - 1's buffer free
        if constexpr (CK) {
            // T after the entries in front of this batch, and the colour of the
            // segment that ends here (only read back for pixels whose last
            // contributor lies behind this point, which are not done)
            if (b > 0 && b % ck_b == 0) {
                ++nck;
                rv.ck[(ck_base + (size_t)nck) * GS2_TILE_PIX + lp] = make_float4(T, c0, c1, c2);
                c0 = c1 = c2 = 0.f;
            }
        }
        if (b + 1 < nbat) {
            issue(b + 1, knext);
            const int j2 = (b + 2) * GS2_TILE_PIX + t;
            if (j2 < n) knext = ids[r.x + j2];
        }
        const int buf = b & 1, b0 = b * GS2_TILE_PIX;
        const int m = min(GS2_TILE_PIX, n - b0);
        // one list entry that lies in the pixel's support (q <= l): composite or stop
        auto composite = [&](int i, float q) {
            const float4 B = sB[buf][i];
            const float alpha = q < B.w ? amax : __fmul_rn(B.y, gs2_falloff(q));
            const float tt = __fmul_rn(T, __fsub_rn(1.f, alpha));
            if (tt < tmin) {
                done = true;
                return;
            }
            const float4 C = sC[buf][i];
            const float wgt = alpha * T;
            c0 = fmaf(wgt, C.x, c0);
            c1 = fmaf(wgt, C.y, c1);
            c2 = fmaf(wgt, C.z, c2);
            T = tt;
            lastc = (uint32_t)(b0 + i + 1);
        };
        // four entries at a time: their quadratic forms do not depend on one
        // another, so their loads and arithmetic overlap; the composites
        // then follow in list order (the same operations as one at a time)
        int i = 0;
        for (; i + 4 <= m && !done; i += 4) {
            float q[4];
            uint32_t hit = 0u;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 A = sA[buf][i + u];
                const float2 Bxz = make_float2(sB[buf][i + u].x, sB[buf][i + u].z);
                q[u] = dec_quad(A.z, A.w, Bxz.x, __fsub_rn(fx, A.x), __fsub_rn(fy, A.y));
                hit |= (q[u] <= Bxz.y) ? 1u << u : 0u;   // sigma G >= alpha_min
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (!done && (hit >> u & 1u)) composite(i + u, q[u]);
        }
        for (; i < m && !done; ++i) {
            const float4 A = sA[buf][i];
            const float2 Bxz = make_float2(sB[buf][i].x, sB[buf][i].z);
            const float q = dec_quad(A.z, A.w, Bxz.x, __fsub_rn(fx, A.x), __fsub_rn(fy, A.y));
            if (q <= Bxz.y) composite(i, q);
        }
    }
    if constexpr (CK) {
        // checkpoint j: (T(c_j), colour of [c_j, end)), summed from the back
        // over this thread's own checkpoints (it wrote them: no barrier).  The
        // accumulation reads checkpoint j of this pixel only if its last
        // contributor lies behind c_j (j <= jmax); the segments from c_{jmax+1}
        // on add no colour, so the sum starts at slot jmax + 1.
        const int jmax = lastc ? min(nck, (int)((lastc - 1u) / (uint32_t)rv.ck_every)) : 0;
        float b0 = 0.f, b1 = 0.f, b2 = 0.f;
        if (jmax == nck) {   // the last segment holds the last contributor
            b0 = c0;
            b1 = c1;
            b2 = c2;
        }
        float4 *base = rv.ck + ck_base * GS2_TILE_PIX + lp;
        // four slots loaded at once: (T(c_j), colour of [c_{j-1}, c_j))
        for (int j = min(nck, jmax + 1); j >= 1; j -= 4) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                v[u] = j - u >= 1 ? base[(size_t)(j - u) * GS2_TILE_PIX] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (j - u >= 1 && j - u <= jmax) base[(size_t)(j - u) * GS2_TILE_PIX] = make_float4(v[u].x, b0, b1, b2);
                b0 += v[u].y;
                b1 += v[u].z;
                b2 += v[u].w;
            }
        }
        c0 = b0;   // the pixel's colour
        c1 = b1;
        c2 = b2;
        // the tile's walk length
        const uint32_t wm = __reduce_max_sync(0xFFFFFFFFu, lastc);
        if (t == 0) sMax = 0u;
        __syncthreads();
        if ((t & 31) == 0) atomicMax(&sMax, wm);
        __syncthreads();
        if (t == 0) rv.tile_maxlast[tile] = sMax;
    }
    if (inside) {
        const size_t P = (size_t)W * H, p = (size_t)py * W + px;
        image[p] = c0;
        image[P + p] = c1;
        image[2 * P + p] = c2;
        rv.tfinal[p] = T;
        rv.last[p] = lastc;
    }
}

cudaError_t launch_raster(gs2_ctx *ctx, ProjView pv, const DevCam &cam, const gs2_config &cfg, float *image,
                          RasterView rv, cudaStream_t st) {
    const unsigned grid = (unsigned)(ctx->tiles_x * ctx->tiles_y);
    if (rv.ck && rv.tile_maxlast && rv.ck_every >= GS2_TILE_PIX)
        k_raster<true><<<grid, GS2_TILE_PIX, 0, st>>>(ctx->ranges, ctx->list_ids, pv, cam.w, cam.h, ctx->tiles_x,
                                                      cfg.alpha_min, cfg.alpha_max, cfg.t_min, image, rv,
                                                      ctx->tile_order);
    else
        k_raster<false><<<grid, GS2_TILE_PIX, 0, st>>>(ctx->ranges, ctx->list_ids, pv, cam.w, cam.h, ctx->tiles_x,
                                                       cfg.alpha_min, cfg.alpha_max, cfg.t_min, image, rv,
                                                       ctx->tile_order);
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError();
}
