// gs2_project: one thread per Gaussian (Sec. 3; App. A.1-A.3).
//
// Per Gaussian: camera-space centre t = Wr p + w, pixel centre
// pi = (fx tx/tz + cx, fy ty/tz + cy), EWA covariance
// Sigma2D = J Wr R diag(s^2) R^T Wr^T J^T + lowpass I with J the perspective
// Jacobian at t (tx/tz, ty/tz clamped to 1.3x the half field of view, the
// standard 3DGS frustum clamp), its inverse (conic), SH colour c~ = sum_i c_i B_i Phi_i(r)
// with r the unit camera->centre direction, the tile rectangle of the support
// { sigma G >= alpha_min } and the depth key.
//
// Memory: reads 13 + 3S floats per Gaussian from planar SoA rows (coalesced
// 4-byte loads across the warp), writes 3 float4 records + rect + counts per
// view.  HBM-bound; FP64 is used only for the depth key (4 DFMA-equivalent
// ops).  One launch projects up to GS2_PROJ_VIEWS views of the same scene
// (the views of a sweep group): the parameters are read once, so four views
// cost 244 + 4 x 68 bytes per Gaussian instead of 4 x (244 + 68).  The
// covariance, conic, thresholds and support box come from the reproducible
// FP32 projection of decide.cuh (explicitly rounded operations only).  The kernel is instantiated per SH
// count S, so every parameter load of a visible Gaussian (4 + 3 + 3S rows) is
// unrolled and issued before the arithmetic: a warp keeps all of them in
// flight at once instead of meeting the memory latency once per loop
// iteration.
#include "common.cuh"
#include "sh.cuh"

__device__ __forceinline__ void write_invisible(const ProjView &pv, int k) {
    pv.touched[k] = 0u;
    pv.rect[k] = make_uint2(0u, 0u);
    pv.recA[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    pv.recB[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    pv.col[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    pv.k2[k] = 0.f;
}

// depth along the view axis: FP64, fixed summation order (products of FP32
// values are exact in FP64, so the key, rounded to FP32, is reproducible bit
// for bit)
__device__ __forceinline__ double view_depth(const DevCam &cam, float px, float py, float pz) {
    double d = (double)cam.V[8] * (double)px;
    d = d + (double)cam.V[9] * (double)py;
    d = d + (double)cam.V[10] * (double)pz;
    return d + (double)cam.V[11];
}

// One visible Gaussian in one view: EWA covariance, conic, thresholds and tile
// rectangle by the reproducible FP32 projection of decide.cuh, then the
// view-dependent colour; writes its records.
template <int S>
__device__ __forceinline__ void project_one(const DevCam &cam, const ProjView &pv, int k, float px, float py, float pz,
                                            float tz, float sigma, const float (&q)[4], const float (&s)[3],
                                            const float (&shc)[3 * S], float lowpass, float alpha_min,
                                            float alpha_max) {
    const DecRec d = dec_project(cam.V, cam.fx, cam.fy, cam.cx, cam.cy, cam.Lx, cam.Ly, px, py, pz, tz, q[0], q[1],
                                 q[2], q[3], s[0], s[1], s[2], sigma, lowpass, alpha_min, alpha_max);
    // tile rectangle of the padded support box (exclusive ends)
    const float fx0 = fmaxf(ceilf(__fsub_rn(d.px, d.rx)), 0.f);
    const float fx1 = fminf(floorf(__fadd_rn(d.px, d.rx)), (float)(cam.w - 1));
    const float fy0 = fmaxf(ceilf(__fsub_rn(d.py, d.ry)), 0.f);
    const float fy1 = fminf(floorf(__fadd_rn(d.py, d.ry)), (float)(cam.h - 1));
    uint32_t touched = 0u;
    uint2 rect = make_uint2(0u, 0u);
    if (fx0 <= fx1 && fy0 <= fy1) {
        const uint32_t tx0 = (uint32_t)fx0 / GS2_TILE, tx1 = (uint32_t)fx1 / GS2_TILE + 1u;
        const uint32_t ty0 = (uint32_t)fy0 / GS2_TILE, ty1 = (uint32_t)fy1 / GS2_TILE + 1u;
        touched = (tx1 - tx0) * (ty1 - ty0);
        rect = make_uint2(tx0 | (ty0 << 16), tx1 | (ty1 << 16));
    }
    pv.touched[k] = touched;
    pv.rect[k] = rect;

    // view-dependent colour
    float rxv = px - cam.o[0], ryv = py - cam.o[1], rzv = pz - cam.o[2];
    const float rn = rsqrtf(rxv * rxv + ryv * ryv + rzv * rzv);
    rxv *= rn; ryv *= rn; rzv *= rn;
    float phi[GS2_MAX_SH];
    sh_phi(S, rxv, ryv, rzv, phi);
    float col[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < S; ++i) acc = fmaf(sh_norm(i) * phi[i], shc[c * S + i], acc);
        col[c] = acc;
    }
    pv.recA[k] = make_float4(d.px, d.py, d.ca, d.cb);
    pv.recB[k] = make_float4(d.cc, sigma, d.l, d.lmax);
    pv.col[k] = make_float4(col[0], col[1], col[2], d.ry);
    pv.k2[k] = d.k2;
}

template <int S>
__global__ void __launch_bounds__(256) k_project(DevScene sc, ProjViews views, float lowpass, float near_z,
                                                 float alpha_min, float alpha_max,
                                                 uint32_t *__restrict__ status) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= sc.n) return;
    const int n = sc.n, nv = views.nv;
    const float px = sc.mean[k], py = sc.mean[n + k], pz = sc.mean[2 * n + k];
    const float sigma = sc.opacity[k];
    // a non-finite parameter makes the Gaussian invisible and raises the
    // status bit; the rest of the view is unaffected (rotation and scales are
    // checked below, once they are loaded for a Gaussian in front of a camera)
    const bool finite = isfinite(px) && isfinite(py) && isfinite(pz) && isfinite(sigma);
    if (!finite && status) atomicOr(status, GS2_ST_NONFINITE);
    float tz[GS2_PROJ_VIEWS];
    bool vis[GS2_PROJ_VIEWS], any = false;
#pragma unroll
    for (int v = 0; v < GS2_PROJ_VIEWS; ++v) {
        vis[v] = false;
        if (v < nv) {
            const double d = view_depth(views.cam[v], px, py, pz);
            tz[v] = (float)d;
            views.pv[v].key[k] = __float_as_uint(tz[v]);
            vis[v] = finite && (d >= (double)near_z) && (sigma >= alpha_min);
            any = any || vis[v];
        }
    }
    if (!any) {
#pragma unroll
        for (int v = 0; v < GS2_PROJ_VIEWS; ++v)
            if (v < nv) write_invisible(views.pv[v], k);
        return;
    }
    // every remaining parameter load first (independent, all in flight together)
    float shc[3 * S];
#pragma unroll
    for (int i = 0; i < 3 * S; ++i) shc[i] = __ldcs(sc.sh + (size_t)i * n + k);
    const float qw = sc.quat[k], qx = sc.quat[n + k], qy = sc.quat[2 * n + k], qz = sc.quat[3 * n + k];
    const float s0 = sc.scale[k], s1 = sc.scale[n + k], s2 = sc.scale[2 * n + k];
    if (!(isfinite(qw) && isfinite(qx) && isfinite(qy) && isfinite(qz) && isfinite(s0) && isfinite(s1) &&
          isfinite(s2))) {
        if (status) atomicOr(status, GS2_ST_NONFINITE);
#pragma unroll
        for (int v = 0; v < GS2_PROJ_VIEWS; ++v)
            if (v < nv) write_invisible(views.pv[v], k);
        return;
    }
    const float qv[4] = {qw, qx, qy, qz}, sv[3] = {s0, s1, s2};
    for (int v = 0; v < GS2_PROJ_VIEWS; ++v) {
        if (v >= nv) break;
        if (vis[v])
            project_one<S>(views.cam[v], views.pv[v], k, px, py, pz, tz[v], sigma, qv, sv, shc, lowpass, alpha_min,
                           alpha_max);
        else
            write_invisible(views.pv[v], k);
    }
}

cudaError_t launch_project_views(const DevScene &sc, const ProjViews &views, const gs2_config &cfg, cudaStream_t st,
                                 uint32_t *status) {
    if (sc.n == 0 || views.nv == 0) return cudaSuccess;
    const unsigned grid = (sc.n + 255) / 256;
    switch (sc.S) {
    case 1: k_project<1><<<grid, 256, 0, st>>>(sc, views, cfg.lowpass, cfg.near_z, cfg.alpha_min, cfg.alpha_max, status); break;
    case 4: k_project<4><<<grid, 256, 0, st>>>(sc, views, cfg.lowpass, cfg.near_z, cfg.alpha_min, cfg.alpha_max, status); break;
    case 9: k_project<9><<<grid, 256, 0, st>>>(sc, views, cfg.lowpass, cfg.near_z, cfg.alpha_min, cfg.alpha_max, status); break;
    default: k_project<16><<<grid, 256, 0, st>>>(sc, views, cfg.lowpass, cfg.near_z, cfg.alpha_min, cfg.alpha_max, status); break;
    }
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError();
}

cudaError_t launch_project(const DevScene &sc, const DevCam &cam, const gs2_config &cfg, ProjView pv, int tiles_x,
                           int tiles_y, cudaStream_t st, uint32_t *status) {
    (void)tiles_x;
    (void)tiles_y;
    ProjViews views;
    views.nv = 1;
    views.cam[0] = cam;
    views.pv[0] = pv;
    return launch_project_views(sc, views, cfg, st, status);
}
