// gs2_loss_derivs: per-pixel e = dL/dc and h = d2L/dc_q^2 (pixel diagonal) of
// L = L2 + lambda L_SSIM (Sec. 4.2 loss equations), fused in one pass.
//
// For window centre p and pixel q (weight w_pq of the 11x11 Gaussian window):
//   dSSIM_p/dc_q   = w_pq (A_p + B_p c^t_q + C_p c_q)
//   d2SSIM_p/dc_q2 = w_pq^2 (K0_p + Kc_p c_q + Kt_p c^t_q + Kct_p c_q c^t_q + Kcc_p c_q^2) + w_pq C_p
// (exact differentiation of f0 f1 / (f2 f3) with the window moments; the
// coefficients depend only on p), so the sums over all windows containing q
// are separable 11-tap correlations of eight coefficient maps with w or w^2.
//
// One CTA owns a 32x16 output tile and keeps everything in shared memory:
// inputs with a 10-pixel halo (52x36), horizontal moment sums, the
// coefficient maps on the 42x26 window-centre region and their horizontal
// correlations.  Each buffer reuses the space of one that is dead by then
// (inputs and coefficient maps share one region, moment sums and correlated
// maps the other): 65 KB, so three CTAs fit on an SM.  HBM traffic per
// pixel: read c, c^t (24 B), write e, h (24 B); the final pass re-reads its
// pixel's c, c^t from L2.
// The correlations run on f32x2 pairs (packed FP32 mul/fma, each half rounded
// as its scalar counterpart): the inputs are kept as (c, c^t) pairs, the
// moment sums as (x, y) and (xx, yy) pair planes beside the xy plane, and the
// eight coefficient maps as four pair planes (A, B), (C, K0), (Kc, Kt),
// (Kct, Kcc) correlated with (w, w), (w, w^2), (w^2, w^2), (w^2, w^2).
#include <mutex>

#include "common.cuh"

#define LT_W 32
#define LT_H 16
#define LRAD 5
#define LWIN 11
#define IN_W (LT_W + 4 * LRAD)
#define IN_H (LT_H + 4 * LRAD)
#define MO_W (LT_W + 2 * LRAD)
#define MO_H (LT_H + 2 * LRAD)
#define SM_IN (IN_W * IN_H)
#define SM_H1 (5 * IN_H * MO_W)
#define SM_K (8 * MO_H * MO_W)
#define SM_R2 (2 * SM_IN > SM_K ? 2 * SM_IN : SM_K)
#define SSIM_SMEM_FLOATS (SM_H1 + SM_R2)

struct SsimConst {
    float g[LWIN];
    float g2[LWIN];
    float c1, c2, lam, scale;
};

__device__ __forceinline__ void block_add_double(double v, double *dst, double *sred) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sred[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sred[i];
        atomicAdd(dst, s);
    }
}

__global__ void __launch_bounds__(256, 3) k_ssim(const float *__restrict__ img, const float *__restrict__ tgt, int W,
                                              int H, SsimConst K, float *__restrict__ eo, float *__restrict__ ho,
                                              double *loss, uint32_t *__restrict__ status) {
    extern __shared__ float sm[];
    // region 1: moment sums, then (once they are consumed) the correlated maps;
    // region 2: the inputs, then (once the moments are formed) the coefficient maps
    float2 *sXY = reinterpret_cast<float2 *>(sm + SM_H1);           // (c, c^t) [IN_H][IN_W]
    float2 *sH01 = reinterpret_cast<float2 *>(sm);                  // (w * x, w * y) [IN_H][MO_W]
    float2 *sH23 = sH01 + IN_H * MO_W;                              // (w * xx, w * yy)
    float *sH4 = reinterpret_cast<float *>(sH23 + IN_H * MO_W);     // w * xy
    float2 *sK2 = reinterpret_cast<float2 *>(sm + SM_H1);           // 4 coefficient pair planes [MO_H][MO_W]
    float2 *sHC2 = reinterpret_cast<float2 *>(sm);                  // 4 correlated pair planes [MO_H][LT_W]
    __shared__ double sred[8];
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * LT_W, y0 = blockIdx.y * LT_H;
    const size_t P = (size_t)W * H;
    double l2acc = 0.0, lsacc = 0.0;
    // window weights of the coefficient pair planes: (w, w), (w, w^2), (w^2, w^2), (w^2, w^2)
    auto cw = [&](int qq, int d) {
        return make_float2(qq < 2 ? K.g[d] : K.g2[d], qq == 0 ? K.g[d] : K.g2[d]);
    };
    for (int c = 0; c < 3; ++c) {
        const float *X = img + c * P, *Y = tgt + c * P;
        {
            // every load of this thread first, then the stores (the loads overlap)
            constexpr int PER = (SM_IN + 255) / 256;
            float xv[PER], yv[PER];
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int i = t + 256 * u;
                const int r = i / IN_W, q = i % IN_W;
                const int gx = x0 - 2 * LRAD + q, gy = y0 - 2 * LRAD + r;
                const bool in = i < SM_IN && gx >= 0 && gx < W && gy >= 0 && gy < H;
                xv[u] = in ? X[(size_t)gy * W + gx] : 0.f;
                yv[u] = in ? Y[(size_t)gy * W + gx] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int i = t + 256 * u;
                if (i >= SM_IN) break;
                float xx = xv[u], yy = yv[u];
                // a non-finite pixel counts as 0 and raises the status bit
                if (!(isfinite(xx) && isfinite(yy))) {
                    if (status) atomicOr(status, GS2_ST_NONFINITE);
                    xx = isfinite(xx) ? xx : 0.f;
                    yy = isfinite(yy) ? yy : 0.f;
                }
                sXY[i] = make_float2(xx, yy);
            }
        }
        __syncthreads();
        // horizontal window sums of x, y, xx, yy, xy: a thread slides one
        // window along HR consecutive outputs of a row (inputs read once)
        constexpr int HR = 6, HSEG = MO_W / HR;   // 42 = 7 x 6
        for (int i = t; i < IN_H * HSEG; i += 256) {
            const int r = i / HSEG, j0 = (i % HSEG) * HR;
            const float2 *xr = sXY + r * IN_W + j0;
            float2 xy[HR + LWIN - 1];
#pragma unroll
            for (int d = 0; d < HR + LWIN - 1; ++d) xy[d] = xr[d];
#pragma unroll
            for (int o = 0; o < HR; ++o) {
                float2 ab = make_float2(0.f, 0.f), sq = ab;
                float cxy = 0.f;
#pragma unroll
                for (int d = 0; d < LWIN; ++d) {
                    const float2 w = make_float2(K.g[d], K.g[d]), v = xy[o + d];
                    const float2 wv = __fmul2_rn(w, v);
                    ab = __ffma2_rn(w, v, ab);
                    sq = __ffma2_rn(wv, v, sq);
                    cxy = fmaf(wv.x, v.y, cxy);
                }
                const int q = r * MO_W + j0 + o;
                sH01[q] = ab;
                sH23[q] = sq;
                sH4[q] = cxy;
            }
        }
        __syncthreads();
        // vertical sums -> moments -> per-centre coefficients: a thread slides
        // down VR consecutive window centres of a column
        constexpr int VR = 4, VSEG = (MO_H + VR - 1) / VR;   // 26 rows in 7 runs
        for (int i = t; i < MO_W * VSEG; i += 256) {
            const int j = i % MO_W, r0 = (i / MO_W) * VR;
            const int nr = min(VR, MO_H - r0);
            float2 mab[VR], msq[VR];
            float mxy[VR];
#pragma unroll
            for (int o = 0; o < VR; ++o) {
                mab[o] = msq[o] = make_float2(0.f, 0.f);
                mxy[o] = 0.f;
            }
#pragma unroll
            for (int d = 0; d < VR + LWIN - 1; ++d) {
                if (r0 + d >= IN_H) break;
                const int q = (r0 + d) * MO_W + j;
                const float2 hab = sH01[q], hsq = sH23[q];
                const float hxy = sH4[q];
#pragma unroll
                for (int o = 0; o < VR; ++o) {
                    const int tap = d - o;
                    if (tap >= 0 && tap < LWIN) {
                        const float2 w = make_float2(K.g[tap], K.g[tap]);
                        mab[o] = __ffma2_rn(w, hab, mab[o]);
                        msq[o] = __ffma2_rn(w, hsq, msq[o]);
                        mxy[o] = fmaf(K.g[tap], hxy, mxy[o]);
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < VR; ++o) {
                if (o >= nr) break;
                const int r = r0 + o;
                const int gx = x0 - LRAD + j, gy = y0 - LRAD + r;
                float co[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
                    const float mu = mab[o].x, mt = mab[o].y;
                    const float var = msq[o].x - mu * mu, vart = msq[o].y - mt * mt, cov = mxy[o] - mu * mt;
                    const float f0 = 2.f * mu * mt + K.c1, f1 = 2.f * cov + K.c2;
                    const float f2 = mu * mu + mt * mt + K.c1, f3 = var + vart + K.c2;
                    const float D = f2 * f3, N = f0 * f1;
                    const float iD = 1.f / D, iD2 = iD * iD, iD3 = iD2 * iD;
                    const float d10 = f1 - f0, d32 = f3 - f2;
                    co[0] = 2.f * mt * d10 * iD - 2.f * N * mu * d32 * iD2;                       // A
                    co[1] = 2.f * f0 * iD;                                                        // B
                    co[2] = -2.f * N * f2 * iD2;                                                  // C
                    co[3] = -8.f * mt * mt * iD - 8.f * mt * mu * d10 * d32 * iD2                 // K0
                            - N * (2.f * f3 - 2.f * f2 - 8.f * mu * mu) * iD2 + 8.f * N * mu * mu * d32 * d32 * iD3;
                    co[4] = -8.f * mt * d10 * f2 * iD2 - 8.f * N * mu * iD2 + 16.f * N * mu * d32 * f2 * iD3;  // Kc
                    co[5] = 8.f * mt * iD - 8.f * f0 * mu * d32 * iD2;                            // Kt
                    co[6] = -8.f * f0 * f2 * iD2;                                                 // Kct
                    co[7] = 8.f * N * f2 * f2 * iD3;                                              // Kcc
                    if (j >= LRAD && j < LRAD + LT_W && r >= LRAD && r < LRAD + LT_H) lsacc += 1.0 - (double)(N * iD);
                }
#pragma unroll
                for (int qq = 0; qq < 4; ++qq)
                    sK2[qq * MO_H * MO_W + r * MO_W + j] = make_float2(co[2 * qq], co[2 * qq + 1]);
            }
        }
        __syncthreads();
        // horizontal correlation of the coefficient pair planes, CR
        // consecutive outputs of a row per thread
        constexpr int CR = 8, CSEG = LT_W / CR;   // 32 = 4 x 8
        for (int i = t; i < 4 * MO_H * CSEG; i += 256) {
            const int qq = i / (MO_H * CSEG), rem = i % (MO_H * CSEG);
            const int r = rem / CSEG, j0 = (rem % CSEG) * CR;
            const float2 *src = sK2 + qq * MO_H * MO_W + r * MO_W + j0;
            float2 v[CR + LWIN - 1];
#pragma unroll
            for (int d = 0; d < CR + LWIN - 1; ++d) v[d] = src[d];
            float2 wt[LWIN];
#pragma unroll
            for (int d = 0; d < LWIN; ++d) wt[d] = cw(qq, d);
#pragma unroll
            for (int o = 0; o < CR; ++o) {
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int d = 0; d < LWIN; ++d) acc = __ffma2_rn(wt[d], v[o + d], acc);
                sHC2[qq * MO_H * LT_W + r * LT_W + j0 + o] = acc;
            }
        }
        __syncthreads();
        // vertical correlation and the per-pixel derivatives: a thread slides
        // down OR output rows of a column
        constexpr int OR = 2, OSEG = LT_H / OR;   // 16 = 8 x 2
        for (int i = t; i < LT_W * OSEG; i += 256) {
            const int j = i % LT_W, r0 = (i / LT_W) * OR;
            float2 v2[OR][4];
#pragma unroll
            for (int o = 0; o < OR; ++o)
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) v2[o][qq] = make_float2(0.f, 0.f);
#pragma unroll
            for (int d = 0; d < OR + LWIN - 1; ++d) {
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    const float2 hv = sHC2[qq * MO_H * LT_W + (r0 + d) * LT_W + j];
#pragma unroll
                    for (int o = 0; o < OR; ++o) {
                        const int tap = d - o;
                        if (tap >= 0 && tap < LWIN) v2[o][qq] = __ffma2_rn(cw(qq, tap), hv, v2[o][qq]);
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < OR; ++o) {
            const int r = r0 + o;
            const int gx = x0 + j, gy = y0 + r;
            if (gx >= W || gy >= H) continue;
            const size_t p = (size_t)c * P + (size_t)gy * W + gx;
            float x = __ldg(img + p), y = __ldg(tgt + p);   // sanitised as in the staging pass
            x = isfinite(x) ? x : 0.f;
            y = isfinite(y) ? y : 0.f;
            const float vo[8] = {v2[o][0].x, v2[o][0].y, v2[o][1].x, v2[o][1].y,
                                 v2[o][2].x, v2[o][2].y, v2[o][3].x, v2[o][3].y};
            const float dS = vo[0] + y * vo[1] + x * vo[2];
            const float d2S = vo[3] + x * vo[4] + y * vo[5] + x * y * vo[6] + x * x * vo[7] + vo[2];
            eo[p] = K.scale * (x - y) - K.lam * K.scale * dS;
            ho[p] = K.scale - K.lam * K.scale * d2S;
            l2acc += 0.5 * (double)(x - y) * (double)(x - y);
            }
        }
        __syncthreads();
    }
    if (loss) {
        block_add_double(l2acc * (double)K.scale, &loss[0], sred);
        block_add_double(lsacc * (double)K.scale, &loss[1], sred);
    }
}

__global__ void __launch_bounds__(256) k_l2(const float *__restrict__ img, const float *__restrict__ tgt, size_t P3,
                                            float scale, float *__restrict__ eo, float *__restrict__ ho,
                                            double *loss, uint32_t *__restrict__ status) {
    __shared__ double sred[8];
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P3; i += (size_t)gridDim.x * blockDim.x) {
        float d = img[i] - tgt[i];
        if (!isfinite(d)) {   // a non-finite pixel counts as 0 and raises the status bit
            if (status) atomicOr(status, GS2_ST_NONFINITE);
            d = 0.f;
        }
        eo[i] = scale * d;
        ho[i] = scale;
        acc += 0.5 * (double)d * (double)d;
    }
    if (loss) block_add_double(acc * (double)scale, &loss[0], sred);
}

// The SSIM kernel's shared-memory opt-in, set once per process (gs2_create
// calls this, so no first launch happens inside a stream capture).
cudaError_t prepare_loss_kernels() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        err = cudaFuncSetAttribute(k_ssim, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   SSIM_SMEM_FLOATS * (int)sizeof(float));
    });
    return err;
}

cudaError_t launch_loss(const float *image, const float *target, int w, int h, const gs2_config &cfg, float *e,
                        float *hh, double *loss_out, cudaStream_t st, uint32_t *status) {
    const size_t P = (size_t)w * h;
    if (P == 0) return cudaSuccess;
    const float scale = (float)(1.0 / (3.0 * (double)P));
    if (cfg.lambda_ssim == 0.f) {
        const size_t P3 = 3 * P;
        int grid = (int)std::min<size_t>((P3 + 255) / 256, 148 * 16);
        k_l2<<<grid, 256, 0, st>>>(image, target, P3, scale, e, hh, loss_out, status);
        GS2_COUNT_LAUNCH(1);
        return cudaGetLastError();
    }
    SsimConst K;
    double g[LWIN], s = 0.0;
    for (int i = 0; i < LWIN; ++i) {
        const double x = i - LRAD;
        g[i] = exp(-x * x / (2.0 * (double)cfg.ssim_sigma * (double)cfg.ssim_sigma));
        s += g[i];
    }
    for (int i = 0; i < LWIN; ++i) {
        K.g[i] = (float)(g[i] / s);
        K.g2[i] = (float)((g[i] / s) * (g[i] / s));
    }
    K.c1 = cfg.ssim_c1;
    K.c2 = cfg.ssim_c2;
    K.lam = cfg.lambda_ssim;
    K.scale = scale;
    const int smem = SSIM_SMEM_FLOATS * (int)sizeof(float);
    const cudaError_t e0 = prepare_loss_kernels();
    if (e0 != cudaSuccess) return e0;
    dim3 grid((w + LT_W - 1) / LT_W, (h + LT_H - 1) / LT_H);
    k_ssim<<<grid, 256, smem, st>>>(image, target, w, h, K, e, hh, loss_out, status);
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError();
}
