// Learned step scale for the local Newton steps (an extension: the paper's
// step size is always 1, Sec. 4.2).  A 8-64-64-1 MLP (ReLU, BF16 weights,
// FP32 accumulation) maps per-(Gaussian, group) features of the plain damped
// step d to a scale alpha = 2 sigmoid(y) in (0, 2); the applied step is
// alpha d, kept inside the same trust radii and bounds as the plain step.
//
// Records logged from the plain method (one per Gaussian and group), float
// [GS2_REC_ROWS][n]:
//   rows 0-7  features (below), row 8 phi0,
//   row 9     label alpha* in [0, 2], or -1 where the record is unusable,
//   row 10    phi1.
// The label looks at a loss L_lab along d: phi0 = grad L_lab . d before the
// step, phi1 = grad L_lab . d after every Gaussian of the group took its step
// (so the coupling of the simultaneous updates is included).  alpha* = 0 when
// phi0 >= 0 (d does not descend L_lab: a rejected step), else the minimum of
// the quadratic line model, phi0 / (phi0 - phi1), 2 where that model is not
// convex, clipped to [0, 2].  The logged sweep takes L_lab = the loss summed
// over every training view at full resolution: an increase of that loss is
// the overshoot of Sec. 4.3.  The step "was accepted" (L_lab decreased under
// the line model) exactly when alpha* > 1/2.
//
// Features, from g, H (the group's block), d and the Gaussian's parameters:
//   f0 log10 clamp(d^T H d / (-g . d), 1e-6, 1e6)   (1 for the undamped step)
//   f1 cos(-g, d)
//   f2 log10 max(|d| / u, 1e-12), u = max(s) for position and scaling, else 1
//   f3 sigma
//   f4 clamp(g_p . d / g . d, -4, 4), g_p the primary view's own gradient: the
//      primary's share of the step's predicted decrease (0 if g . d >= 0)
//   f5 1 if a trust radius or bound limits the step (within 1e-3), else 0
//   f6 log10 clamp(|g| / (mean|diag H| |d|), 1e-6, 1e6)
//   f7 group / 4
// A record is usable when |d| > 0, g . d < 0 and every feature is finite.
//
// Parameter layout (GS2_MLP_NPARAM words, BF16 for inference, FP32 master):
//   W1 [64][8], b1 [64], W2 [64][64], b2 [64], W3 [64], b3
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"

#define NF GS2_MLP_NFEAT
#define NH GS2_MLP_HIDDEN
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + NH * NF)
#define OFF_W2 (OFF_B1 + NH)
#define OFF_B2 (OFF_W2 + NH * NH)
#define OFF_W3 (OFF_B2 + NH)
#define OFF_B3 (OFF_W3 + NH)
#define NPARAM (OFF_B3 + 1)
#define RROWS GS2_REC_ROWS

static_assert(NPARAM == GS2_MLP_NPARAM, "parameter count in gs2.h must match the layout");
static_assert(RROWS == NF + 3, "record rows: features, phi0, label, phi1");

// ---------------------------------------------------------------- features
struct StepStats {
    float gd, q, gg, dd, hd;   // g.d, d^T H d, |g|^2, |d|^2, mean |diag H|
    float gpd;                 // g_p . d (primary view's own gradient)
    bool clipped;
};

__device__ __forceinline__ float smax_of(const DevScene &sc, int k) {
    const int n = sc.n;
    return fmaxf(sc.scale[k], fmaxf(sc.scale[n + k], sc.scale[2 * n + k]));
}

__device__ __forceinline__ bool near_or_past(float v, float lim) { return v >= (1.f - 1e-3f) * lim; }

// gp: the primary view's gradient rows [D][n] (position, rotation, scaling,
// opacity; colour takes it from view slot 0 of B)
__device__ StepStats step_stats(int group, const float *__restrict__ B, int n_views, const DevScene &sc, int k,
                                const float *__restrict__ step, const float *__restrict__ gp, const gs2_config &cfg,
                                float smax) {
    const int n = sc.n, S = sc.S;
    StepStats r{};
    if (group == GS2_POS || group == GS2_SCALE) {
        float d[3], g[3];
        for (int i = 0; i < 3; ++i) {
            d[i] = step[(size_t)i * n + k];
            g[i] = B[(size_t)i * n + k];
        }
        const float h00 = B[(size_t)3 * n + k], h01 = B[(size_t)4 * n + k], h02 = B[(size_t)5 * n + k];
        const float h11 = B[(size_t)6 * n + k], h12 = B[(size_t)7 * n + k], h22 = B[(size_t)8 * n + k];
        r.gd = g[0] * d[0] + g[1] * d[1] + g[2] * d[2];
        r.gpd = gp[k] * d[0] + gp[(size_t)n + k] * d[1] + gp[(size_t)2 * n + k] * d[2];
        r.q = h00 * d[0] * d[0] + h11 * d[1] * d[1] + h22 * d[2] * d[2] +
              2.f * (h01 * d[0] * d[1] + h02 * d[0] * d[2] + h12 * d[1] * d[2]);
        r.gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
        r.dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        r.hd = (fabsf(h00) + fabsf(h11) + fabsf(h22)) * (1.f / 3.f);
        if (group == GS2_POS) {
            r.clipped = near_or_past(sqrtf(r.dd), cfg.trust_pos * smax);
        } else {
            for (int i = 0; i < 3; ++i) {
                const float s = sc.scale[(size_t)i * n + k];
                r.clipped |= near_or_past(-d[i], s - s / cfg.scale_trust) || near_or_past(d[i], cfg.scale_trust * s - s);
            }
        }
        return r;
    }
    if (group == GS2_ROT || group == GS2_OPACITY) {
        const float g = B[k], h = B[n + k], d = step[k];
        r.gd = g * d;
        r.gpd = gp[k] * d;
        r.q = h * d * d;
        r.gg = g * g;
        r.dd = d * d;
        r.hd = fabsf(h);
        if (group == GS2_ROT) {
            r.clipped = near_or_past(fabsf(d), cfg.trust_rot);
        } else {
            const float sg = sc.opacity[k], tau = cfg.frac_to_boundary;
            r.clipped = near_or_past(-d, tau * sg) || near_or_past(d, tau * (1.f - sg));
        }
        return r;
    }
    // colour: per channel H_c = sum_v s_cv b_v b_v^T, g_c = sum_v a_cv b_v
    const size_t slot = (size_t)(6 + S) * n;
    float hsum = 0.f;
    for (int c = 0; c < 3; ++c) {
        float dc[16], gc[16], hc[16];
        float dn = 0.f;
        for (int i = 0; i < S; ++i) {
            dc[i] = step[(size_t)(c * S + i) * n + k];
            gc[i] = 0.f;
            hc[i] = 0.f;
            dn += dc[i] * dc[i];
        }
        for (int v = 0; v < n_views; ++v) {
            const float *Bv = B + v * slot;
            const float a = Bv[(size_t)c * n + k], s = Bv[(size_t)(3 + c) * n + k];
            float t = 0.f;
            for (int i = 0; i < S; ++i) {
                const float b = Bv[(size_t)(6 + i) * n + k];
                t += b * dc[i];
                gc[i] += a * b;
                hc[i] += s * b * b;
            }
            r.gd += a * t;
            r.q += s * t * t;
            if (v == 0) r.gpd += a * t;
        }
        for (int i = 0; i < S; ++i) {
            r.gg += gc[i] * gc[i];
            hsum += fabsf(hc[i]);
        }
        r.dd += dn;
        r.clipped |= near_or_past(sqrtf(dn), cfg.trust_color);
    }
    r.hd = hsum / (float)(3 * S);
    return r;
}

__device__ __forceinline__ float clamp_log10(float v, float lo, float hi) { return log10f(fminf(fmaxf(v, lo), hi)); }

// the 8 features; returns whether the record is usable
__device__ bool step_features(int group, const StepStats &st, float sigma, float smax, float f[NF]) {
    const float dn = sqrtf(st.dd), gn = sqrtf(st.gg);
    const float u = (group == GS2_POS || group == GS2_SCALE) ? smax : 1.f;
    const float mgd = -st.gd;
    f[0] = clamp_log10(mgd > 0.f ? st.q / mgd : 1e6f, 1e-6f, 1e6f);
    f[1] = (gn * dn > 0.f) ? mgd / (gn * dn) : 0.f;
    f[2] = log10f(fmaxf(dn / u, 1e-12f));
    f[3] = sigma;
    f[4] = (st.gd < 0.f) ? fminf(fmaxf(st.gpd / st.gd, -4.f), 4.f) : 0.f;
    f[5] = st.clipped ? 1.f : 0.f;
    f[6] = clamp_log10(st.hd * dn > 0.f ? gn / (st.hd * dn) : 1e6f, 1e-6f, 1e6f);
    f[7] = 0.25f * (float)group;
    bool ok = st.dd > 0.f && st.gd < 0.f;
#pragma unroll
    for (int i = 0; i < NF; ++i) ok = ok && isfinite(f[i]);
    return ok;
}

__global__ void __launch_bounds__(128) k_step_records(int group, const float *__restrict__ B, int n_views,
                                                      DevScene sc, const float *__restrict__ step,
                                                      const float *__restrict__ gp, gs2_config cfg,
                                                      float *__restrict__ rec) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = sc.n;
    if (k >= n) return;
    const float smax = smax_of(sc, k);
    const StepStats st = step_stats(group, B, n_views, sc, k, step, gp, cfg, smax);
    float f[NF];
    const bool ok = step_features(group, st, sc.opacity[k], smax, f);
#pragma unroll
    for (int i = 0; i < NF; ++i) rec[(size_t)i * n + k] = f[i];
    rec[(size_t)NF * n + k] = st.gd;
    rec[(size_t)(NF + 1) * n + k] = ok ? 0.f : -1.f;   // label pending (0) or unusable (-1)
    rec[(size_t)(NF + 2) * n + k] = 0.f;
}

// g . d from a block (the after-step block for the labels)
__device__ float block_dot_step(int group, const float *__restrict__ B, int n_views, int n, int S, int k,
                                const float *__restrict__ step) {
    if (group == GS2_POS || group == GS2_SCALE) {
        float r = 0.f;
        for (int i = 0; i < 3; ++i) r += B[(size_t)i * n + k] * step[(size_t)i * n + k];
        return r;
    }
    if (group == GS2_ROT || group == GS2_OPACITY) return B[k] * step[k];
    const size_t slot = (size_t)(6 + S) * n;
    float r = 0.f;
    for (int v = 0; v < n_views; ++v) {
        const float *Bv = B + v * slot;
        for (int c = 0; c < 3; ++c) {
            float t = 0.f;
            for (int i = 0; i < S; ++i) t += Bv[(size_t)(6 + i) * n + k] * step[(size_t)(c * S + i) * n + k];
            r += Bv[(size_t)c * n + k] * t;
        }
    }
    return r;
}

// phi1 from a block accumulated after the step (Bafter, n_views slots) or, if
// phi1 is not NULL, as given; phi0 from row 8
__global__ void __launch_bounds__(128) k_step_labels(int group, const float *__restrict__ Bafter, int n_views,
                                                     DevScene sc, const float *__restrict__ step,
                                                     const float *__restrict__ phi1v, float *__restrict__ rec) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = sc.n;
    if (k >= n) return;
    float *lab = rec + (size_t)(NF + 1) * n + k;
    if (*lab < 0.f) return;
    const float phi0 = rec[(size_t)NF * n + k];
    const float phi1 = phi1v ? phi1v[k] : block_dot_step(group, Bafter, n_views, n, sc.S, k, step);
    rec[(size_t)(NF + 2) * n + k] = phi1;
    const float den = phi0 - phi1;
    float a = (den < 0.f) ? phi0 / den : 2.f;
    if (!(phi0 < 0.f)) a = 0.f;                       // not a descent direction of the label loss
    *lab = isfinite(a) ? fminf(fmaxf(a, 0.f), 2.f) : -1.f;
}

// out[k] += g . d of a one-view block
__global__ void __launch_bounds__(128) k_phi_add(int group, const float *__restrict__ B, DevScene sc,
                                                 const float *__restrict__ step, float *__restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= sc.n) return;
    out[k] += block_dot_step(group, B, 1, sc.n, sc.S, k, step);
}

// ---------------------------------------------------------------- inference
// forward pass of one input; weights (converted to FP32) in shared memory
__device__ __forceinline__ float mlp_eval(const float *__restrict__ sw, const float x[NF]) {
    float h1[NH];
#pragma unroll
    for (int j = 0; j < NH; ++j) {
        float acc = sw[OFF_B1 + j];
#pragma unroll
        for (int i = 0; i < NF; ++i) acc = fmaf(sw[OFF_W1 + j * NF + i], x[i], acc);
        h1[j] = fmaxf(acc, 0.f);
    }
    float y = sw[OFF_B3];
#pragma unroll 2
    for (int j = 0; j < NH; ++j) {
        const float4 *w4 = reinterpret_cast<const float4 *>(sw + OFF_W2 + j * NH);
        float acc = sw[OFF_B2 + j];
#pragma unroll
        for (int q = 0; q < NH / 4; ++q) {
            const float4 w = w4[q];
            acc = fmaf(w.x, h1[4 * q], acc);
            acc = fmaf(w.y, h1[4 * q + 1], acc);
            acc = fmaf(w.z, h1[4 * q + 2], acc);
            acc = fmaf(w.w, h1[4 * q + 3], acc);
        }
        y = fmaf(sw[OFF_W3 + j], fmaxf(acc, 0.f), y);
    }
    return y;
}

__device__ __forceinline__ float scale_of(float y) { return 2.f / (1.f + expf(-y)); }

__device__ __forceinline__ void load_weights(float *sw, const __nv_bfloat16 *__restrict__ w) {
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) sw[i] = __bfloat162float(w[i]);
}

// step <- alpha d inside learned_trust times the plain step's trust radii
// (position, rotation, colour; scale bounds [s / k^lt, k^lt s], lt =
// learned_trust) and the opacity fraction-to-boundary; the plain step stays
// where the record is unusable or alpha is not finite.  With learned_trust > 1
// a step the plain radius clipped can be lengthened (alpha > 1) up to the
// wider radius: where the radii bind, the scale acts as a learned per-Gaussian
// trust radius.
__global__ void __launch_bounds__(128) k_learned_scale(int group, const float *__restrict__ B, int n_views,
                                                       DevScene sc, float *__restrict__ step,
                                                       const float *__restrict__ gp, gs2_config cfg,
                                                       const __nv_bfloat16 *__restrict__ w) {
    __shared__ __align__(16) float sw[NPARAM + 3];
    load_weights(sw, w);
    __syncthreads();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = sc.n, S = sc.S;
    if (k >= n) return;
    const float smax = smax_of(sc, k);
    const StepStats st = step_stats(group, B, n_views, sc, k, step, gp, cfg, smax);
    float f[NF];
    if (!step_features(group, st, sc.opacity[k], smax, f)) return;
    const float a = scale_of(mlp_eval(sw, f));
    if (!isfinite(a)) return;
    const float lt = cfg.learned_trust;
    if (group == GS2_POS) {
        const float lim = lt * cfg.trust_pos * smax, dn = a * sqrtf(st.dd);
        const float m = (dn > lim) ? a * lim / dn : a;
        for (int i = 0; i < 3; ++i) step[(size_t)i * n + k] *= m;
    } else if (group == GS2_SCALE) {
        const float kk = powf(cfg.scale_trust, lt);
        for (int i = 0; i < 3; ++i) {
            const float s = sc.scale[(size_t)i * n + k];
            const float lo = s / kk - s, hi = kk * s - s;
            step[(size_t)i * n + k] = fminf(fmaxf(a * step[(size_t)i * n + k], lo), hi);
        }
    } else if (group == GS2_ROT) {
        step[k] = fminf(fmaxf(a * step[k], -lt * cfg.trust_rot), lt * cfg.trust_rot);
    } else if (group == GS2_OPACITY) {
        const float sg = sc.opacity[k], tau = cfg.frac_to_boundary;
        step[k] = fminf(fmaxf(a * step[k], -tau * sg), tau * (1.f - sg));
    } else {
        for (int c = 0; c < 3; ++c) {
            float dn = 0.f;
            for (int i = 0; i < S; ++i) {
                const float x = step[(size_t)(c * S + i) * n + k];
                dn += x * x;
            }
            dn = a * sqrtf(dn);
            const float m = (dn > lt * cfg.trust_color) ? a * lt * cfg.trust_color / dn : a;
            for (int i = 0; i < S; ++i) step[(size_t)(c * S + i) * n + k] *= m;
        }
    }
}

cudaError_t launch_step_records(int group, const void *blocks, int n_views, const DevScene &sc, const void *step,
                                const float *gp, const gs2_config &cfg, float *rec, cudaStream_t st) {
    if (sc.n == 0) return cudaSuccess;
    k_step_records<<<(sc.n + 127) / 128, 128, 0, st>>>(group, (const float *)blocks, n_views, sc,
                                                      (const float *)step, gp, cfg, rec);
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError();
}

cudaError_t launch_step_labels(int group, const void *blocks_after, int n_views, const DevScene &sc,
                               const void *step, const float *phi1, float *rec, cudaStream_t st) {
    if (sc.n == 0) return cudaSuccess;
    k_step_labels<<<(sc.n + 127) / 128, 128, 0, st>>>(group, (const float *)blocks_after, n_views, sc,
                                                     (const float *)step, phi1, rec);
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError();
}

cudaError_t launch_phi_add(int group, const void *blocks_one_view, const DevScene &sc, const void *step, float *out,
                           cudaStream_t st) {
    if (sc.n == 0) return cudaSuccess;
    k_phi_add<<<(sc.n + 127) / 128, 128, 0, st>>>(group, (const float *)blocks_one_view, sc, (const float *)step,
                                                 out);
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError();
}

cudaError_t launch_learned_scale(int group, const void *blocks, int n_views, const DevScene &sc, void *step,
                                 const float *gp, const gs2_config &cfg, const void *w, cudaStream_t st) {
    if (sc.n == 0 || !w) return cudaSuccess;
    k_learned_scale<<<(sc.n + 127) / 128, 128, 0, st>>>(group, (const float *)blocks, n_views, sc, (float *)step,
                                                       gp, cfg, (const __nv_bfloat16 *)w);
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- learned damping
// A second network of the same shape and the same features predicts, for the
// position, scaling and colour groups (whose damping turns the step, not only
// shortens it), a multiplier rho of the damping mu0 of the Gaussian's solve:
// rho = 10^(1.5 alpha) in (1, 1e3), alpha = 2 sigmoid(y): the damping can only
// grow (measured: applying the all-view best candidate per Gaussian gained
// 1.7-1.8 dB after 30 sweeps on the object workload, of which raising the
// damping gave 1.3-1.5 dB and lowering it 0.4-0.5).  The solve is then
// repeated with mu0 rho.  Its records share the step records' features; the
// label (row 9) is alpha_rho* = 2 log10(rho*) / 3 with rho* the multiplier,
// among 10^0, 10^0.5, .., 10^3, whose damped step (same solve, trust radii and
// bounds) minimises the quadratic model of the loss over every training view,
// Q(d) = g_all . d + 1/2 d^T H_all d; -1 where the step record is unusable, no
// candidate lowers Q, or the group's damping is not learned.
// Rows 8 and 10 turn the label into the line objective's weighted quadratic
// (k_damp_labels), so training can weight each record by how much its choice
// of damping matters.
__device__ __forceinline__ float rho_of(float a) { return exp10f(1.5f * a); }

__global__ void __launch_bounds__(128) k_learned_damping(int group, const float *__restrict__ B, int n_views,
                                                         DevScene sc, const float *__restrict__ step,
                                                         const float *__restrict__ gp, gs2_config cfg,
                                                         const __nv_bfloat16 *__restrict__ w, float *__restrict__ rho) {
    __shared__ __align__(16) float sw[NPARAM + 3];
    load_weights(sw, w);
    __syncthreads();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= sc.n) return;
    const float smax = smax_of(sc, k);
    const StepStats st = step_stats(group, B, n_views, sc, k, step, gp, cfg, smax);
    float f[NF];
    float r = 1.f;
    if (step_features(group, st, sc.opacity[k], smax, f)) {
        const float a = scale_of(mlp_eval(sw, f));
        if (isfinite(a)) r = rho_of(a);
    }
    rho[k] = r;
}

// Q of a candidate step (the damping multiplier rho_j) from the all-view
// blocks; the smallest Q so far and its multiplier are kept (first: set)
__global__ void __launch_bounds__(128) k_damp_eval(int group, const float *__restrict__ Ball, int n_all, DevScene sc,
                                                   const float *__restrict__ step, gs2_config cfg, float rho_j,
                                                   float *__restrict__ best_q, float *__restrict__ best_rho,
                                                   float *__restrict__ worst_q, int first) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= sc.n) return;
    // g_p is not used by Q: the all-view blocks stand in for it
    const StepStats st = step_stats(group, Ball, n_all, sc, k, step, Ball, cfg, smax_of(sc, k));
    float q = st.gd + 0.5f * st.q;
    const bool fin = isfinite(q);
    if (!fin) q = INFINITY;
    if (first || q < best_q[k]) {
        best_q[k] = q;
        best_rho[k] = rho_j;
    }
    if (first) worst_q[k] = fin ? q : -INFINITY;
    else if (fin && q > worst_q[k]) worst_q[k] = q;
}

// rows 8 and 10 hold the weighted quadratic -w a* a + 1/2 w a^2 in the line
// objective's form (phi0 = -w a*, phi1 = phi0 + w): minimal at the label a*,
// weighted by w = the spread of Q over the candidates (how much the choice
// matters); 0 where there is no label
__global__ void __launch_bounds__(128) k_damp_labels(int group, const float *__restrict__ rec,
                                                     const float *__restrict__ best_q,
                                                     const float *__restrict__ worst_q,
                                                     const float *__restrict__ best_rho, int n,
                                                     float *__restrict__ rec_d) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
#pragma unroll
    for (int i = 0; i < NF; ++i) rec_d[(size_t)i * n + k] = rec[(size_t)i * n + k];   // features
    float lab = -1.f, w = 0.f;
    if (damping_learned(group) && best_q && rec[(size_t)(NF + 1) * n + k] >= 0.f && best_q[k] < 0.f) {
        lab = fminf(fmaxf(log10f(best_rho[k]) * (2.f / 3.f), 0.f), 2.f);
        w = fmaxf(worst_q[k] - best_q[k], 0.f);
    }
    rec_d[(size_t)NF * n + k] = -w * lab;
    rec_d[(size_t)(NF + 1) * n + k] = lab;
    rec_d[(size_t)(NF + 2) * n + k] = -w * lab + w;
}

__global__ void k_add_floats(float *__restrict__ dst, const float *__restrict__ src, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        dst[i] += src[i];
}

cudaError_t launch_learned_damping(int group, const void *blocks, int n_views, const DevScene &sc, const void *step,
                                   const float *gp, const gs2_config &cfg, const void *w, float *rho,
                                   cudaStream_t st) {
    if (sc.n == 0 || !w) return cudaSuccess;
    k_learned_damping<<<(sc.n + 127) / 128, 128, 0, st>>>(group, (const float *)blocks, n_views, sc,
                                                         (const float *)step, gp, cfg, (const __nv_bfloat16 *)w, rho);
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError();
}

cudaError_t launch_damp_eval(int group, const void *blocks_all, int n_all, const DevScene &sc, const void *step,
                             const gs2_config &cfg, float rho_j, float *best_q, float *best_rho, float *worst_q,
                             int first, cudaStream_t st) {
    if (sc.n == 0) return cudaSuccess;
    k_damp_eval<<<(sc.n + 127) / 128, 128, 0, st>>>(group, (const float *)blocks_all, n_all, sc,
                                                   (const float *)step, cfg, rho_j, best_q, best_rho, worst_q, first);
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError();
}

cudaError_t launch_damp_labels(int group, const float *rec, const float *best_q, const float *worst_q,
                               const float *best_rho, int n, float *rec_damp, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_damp_labels<<<(n + 127) / 128, 128, 0, st>>>(group, rec, best_q, worst_q, best_rho, n, rec_damp);
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError();
}

cudaError_t launch_add_floats(float *dst, const float *src, size_t count, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    k_add_floats<<<(unsigned)std::min<size_t>((count + 255) / 256, 148 * 8), 256, 0, st>>>(dst, src, count);
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- training
// Loss of a batch, over the usable records (label >= 0):
//   labels:      1/2 sum (alpha(x) - alpha*)^2
//   line model:  sum s_c (phi0 alpha + 1/2 (phi1 - phi0) alpha^2), the change of
//                the label loss that the line model predicts for the step
//                alpha d, with s_c a per-chunk scale (chunk_scale)
// Record r of the batch is idx[r] (or r when idx is NULL) of a record buffer
// made of chunks [RROWS][chunk_n]: row j of record i at
// rec[(i / chunk_n) RROWS chunk_n + j chunk_n + i % chunk_n].
// Persistent grid of GS2_MLP_GRID CTAs; each CTA keeps its gradient partial sum
// in registers over its 64-record tiles and writes it to its own row of the
// partial buffer (no atomics; the sum over rows is taken in a fixed order).
#define TB 64
#define GT 256
#define PPT ((NPARAM + GT - 1) / GT)

struct TileSmem {
    float x[TB][NF];
    float h1[TB][NH + 1], h2[TB][NH + 1], d2[TB][NH + 1], d1[TB][NH + 1];
    float dy[TB], yl[TB], ml[TB], p0[TB], cv[TB];   // label, mask, s phi0, s (phi1 - phi0)
    double red[2][TB];
};

__device__ __forceinline__ const float *record_base(const float *__restrict__ rec, int64_t chunk_n,
                                                   const int64_t *__restrict__ idx, int64_t r, int64_t *chunk) {
    const int64_t i = idx ? idx[r] : r;
    *chunk = i / chunk_n;
    return rec + (i / chunk_n) * RROWS * chunk_n + (i % chunk_n);
}

__device__ __forceinline__ void load_record(const float *__restrict__ rec, int64_t chunk_n,
                                            const int64_t *__restrict__ idx, int64_t r, float x[NF], float *y) {
    int64_t c;
    const float *base = record_base(rec, chunk_n, idx, r, &c);
#pragma unroll
    for (int j = 0; j < NF; ++j) x[j] = base[j * chunk_n];
    *y = base[(NF + 1) * chunk_n];
}

__global__ void __launch_bounds__(GT) k_mlp_grad(const __nv_bfloat16 *__restrict__ w, const float *__restrict__ rec,
                                                 int64_t chunk_n, const int64_t *__restrict__ idx, int64_t nrec,
                                                 const float *__restrict__ chunk_scale, float *__restrict__ partial,
                                                 double *__restrict__ stats) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sw = reinterpret_cast<float *>(smem_raw);
    TileSmem &sm = *reinterpret_cast<TileSmem *>(smem_raw + sizeof(float) * ((NPARAM + 3) & ~3));
    const int t = threadIdx.x;
    load_weights(sw, w);
    float acc[PPT];
#pragma unroll
    for (int m = 0; m < PPT; ++m) acc[m] = 0.f;
    double lsum = 0.0, cnt = 0.0;
    const int64_t ntiles = (nrec + TB - 1) / TB;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        const int64_t r0 = tile * TB;
        if (t < TB) {
            float x[NF], y = -1.f, p0 = 0.f, cv = 0.f;
            bool use = false;
            if (r0 + t < nrec) {
                int64_t c;
                const float *base = record_base(rec, chunk_n, idx, r0 + t, &c);
#pragma unroll
                for (int j = 0; j < NF; ++j) x[j] = base[j * chunk_n];
                y = base[(NF + 1) * chunk_n];
                use = y >= 0.f;
#pragma unroll
                for (int j = 0; j < NF; ++j) use = use && isfinite(x[j]);
                if (chunk_scale) {
                    const float sc = chunk_scale[c], f0 = base[NF * chunk_n], f1 = base[(NF + 2) * chunk_n];
                    p0 = sc * f0;
                    cv = sc * (f1 - f0);
                    use = use && isfinite(p0) && isfinite(cv);
                }
            }
#pragma unroll
            for (int j = 0; j < NF; ++j) sm.x[t][j] = use ? x[j] : 0.f;
            sm.yl[t] = use ? y : 0.f;
            sm.ml[t] = use ? 1.f : 0.f;
            sm.p0[t] = use ? p0 : 0.f;
            sm.cv[t] = use ? cv : 0.f;
        }
        __syncthreads();
        for (int i = t; i < TB * NH; i += GT) {      // layer 1
            const int r = i / NH, j = i % NH;
            float s = sw[OFF_B1 + j];
#pragma unroll
            for (int c = 0; c < NF; ++c) s = fmaf(sw[OFF_W1 + j * NF + c], sm.x[r][c], s);
            sm.h1[r][j] = fmaxf(s, 0.f);
        }
        __syncthreads();
        for (int i = t; i < TB * NH; i += GT) {      // layer 2
            const int r = i / NH, j = i % NH;
            float s = sw[OFF_B2 + j];
#pragma unroll 16
            for (int c = 0; c < NH; ++c) s = fmaf(sw[OFF_W2 + j * NH + c], sm.h1[r][c], s);
            sm.h2[r][j] = fmaxf(s, 0.f);
        }
        __syncthreads();
        if (t < TB) {                                // output, loss, dL/dy
            float y = sw[OFF_B3];
            for (int c = 0; c < NH; ++c) y = fmaf(sw[OFF_W3 + c], sm.h2[t][c], y);
            const float a = scale_of(y);
            float dlda;                              // dL/d alpha
            if (chunk_scale) {
                lsum += (double)sm.ml[t] * ((double)sm.p0[t] * a + 0.5 * (double)sm.cv[t] * a * a);
                dlda = (sm.p0[t] + sm.cv[t] * a) * sm.ml[t];
            } else {
                const float e = (a - sm.yl[t]) * sm.ml[t];
                lsum += 0.5 * (double)e * (double)e;
                dlda = e;
            }
            cnt += (double)sm.ml[t];
            sm.dy[t] = dlda * a * (1.f - 0.5f * a);  // d alpha / dy = alpha (1 - alpha / 2)
        }
        __syncthreads();
        for (int i = t; i < TB * NH; i += GT) {      // through layer 3 and the second ReLU
            const int r = i / NH, j = i % NH;
            sm.d2[r][j] = (sm.h2[r][j] > 0.f) ? sm.dy[r] * sw[OFF_W3 + j] : 0.f;
        }
        __syncthreads();
        for (int i = t; i < TB * NH; i += GT) {      // through layer 2 and the first ReLU
            const int r = i / NH, c = i % NH;
            float s = 0.f;
#pragma unroll 16
            for (int j = 0; j < NH; ++j) s = fmaf(sw[OFF_W2 + j * NH + c], sm.d2[r][j], s);
            sm.d1[r][c] = (sm.h1[r][c] > 0.f) ? s : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < PPT; ++m) {              // parameter gradients of the tile
            const int i = t + m * GT;
            if (i >= NPARAM) break;
            float s = 0.f;
            if (i < OFF_B1) {
                const int j = i / NF, c = i % NF;
                for (int r = 0; r < TB; ++r) s = fmaf(sm.d1[r][j], sm.x[r][c], s);
            } else if (i < OFF_W2) {
                const int j = i - OFF_B1;
                for (int r = 0; r < TB; ++r) s += sm.d1[r][j];
            } else if (i < OFF_B2) {
                const int j = (i - OFF_W2) / NH, c = (i - OFF_W2) % NH;
                for (int r = 0; r < TB; ++r) s = fmaf(sm.d2[r][j], sm.h1[r][c], s);
            } else if (i < OFF_W3) {
                const int j = i - OFF_B2;
                for (int r = 0; r < TB; ++r) s += sm.d2[r][j];
            } else if (i < OFF_B3) {
                const int c = i - OFF_W3;
                for (int r = 0; r < TB; ++r) s = fmaf(sm.dy[r], sm.h2[r][c], s);
            } else {
                for (int r = 0; r < TB; ++r) s += sm.dy[r];
            }
            acc[m] += s;
        }
    }
    float *row = partial + (size_t)blockIdx.x * NPARAM;
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
        const int i = t + m * GT;
        if (i < NPARAM) row[i] = acc[m];
    }
    __syncthreads();
    if (t < TB) {
        sm.red[0][t] = lsum;
        sm.red[1][t] = cnt;
    }
    for (int o = TB / 2; o > 0; o >>= 1) {
        __syncthreads();
        if (t < o) {
            sm.red[0][t] += sm.red[0][t + o];
            sm.red[1][t] += sm.red[1][t + o];
        }
    }
    if (t == 0) {
        stats[2 * blockIdx.x] = sm.red[0][0];
        stats[2 * blockIdx.x + 1] = sm.red[1][0];
    }
}

static size_t grad_smem_bytes() { return sizeof(float) * ((NPARAM + 3) & ~3) + sizeof(TileSmem); }

__global__ void __launch_bounds__(128) k_mlp_forward(const __nv_bfloat16 *__restrict__ w,
                                                     const float *__restrict__ rec, int64_t chunk_n,
                                                     const int64_t *__restrict__ idx, int64_t nrec,
                                                     float *__restrict__ out) {
    __shared__ __align__(16) float sw[NPARAM + 3];
    load_weights(sw, w);
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrec) return;
    float x[NF], y;
    load_record(rec, chunk_n, idx, r, x, &y);
    out[r] = scale_of(mlp_eval(sw, x));
}

// Adam on the FP32 master weights with the batch mean gradient (partials
// summed in row order, divided by the usable-record count), then the BF16 copy
__global__ void k_mlp_adam(float *__restrict__ master, __nv_bfloat16 *__restrict__ w,
                           const float *__restrict__ partial, int nrows, const double *__restrict__ stats,
                           float *__restrict__ m, float *__restrict__ v, int step, float lr, float b1, float b2,
                           float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    double cnt = 0.0;
    for (int r = 0; r < nrows; ++r) cnt += stats[2 * r + 1];
    if (!(cnt > 0.0)) return;
    float gsum = 0.f;
    for (int r = 0; r < nrows; ++r) gsum += partial[(size_t)r * NPARAM + i];
    const float gi = (float)((double)gsum / cnt);
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(b1, (float)step));
    const float vh = vi / (1.f - powf(b2, (float)step));
    const float p = master[i] - lr * mh / (sqrtf(vh) + eps);
    master[i] = p;
    w[i] = __float2bfloat16_rn(p);
}

extern "C" gs2_status gs2_mlp_forward(const uint16_t *w_bf16, const float *records, int64_t chunk_n,
                                      const int64_t *idx, int64_t nrec, float *out, gs2_stream stream) {
    if (!w_bf16 || !records || !out || nrec < 0 || chunk_n < 1) return GS2_ERR_ARG;
    if (nrec == 0) return GS2_OK;
    k_mlp_forward<<<(unsigned)((nrec + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
        (const __nv_bfloat16 *)w_bf16, records, chunk_n, idx, nrec, out);
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError() == cudaSuccess ? GS2_OK : GS2_ERR_CUDA;
}

// s_c = 1 / sum over the chunk's usable records of |phi0| (0 for none)
__global__ void k_chunk_scale(const float *__restrict__ rec, int64_t chunk_n, float *__restrict__ out) {
    __shared__ double red[256];
    const float *base = rec + (int64_t)blockIdx.x * RROWS * chunk_n;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < chunk_n; i += blockDim.x) {
        const float lab = base[(NF + 1) * chunk_n + i], p0 = base[NF * chunk_n + i];
        if (lab >= 0.f && isfinite(p0)) acc += fabs((double)p0);
    }
    red[threadIdx.x] = acc;
    for (int o = 128; o > 0; o >>= 1) {
        __syncthreads();
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0] > 0.0 ? (float)(1.0 / red[0]) : 0.f;
}

extern "C" gs2_status gs2_records_chunk_scale(const float *records, int64_t chunk_n, int64_t n_chunks, float *out,
                                              gs2_stream stream) {
    if (!records || !out || chunk_n < 1 || n_chunks < 0) return GS2_ERR_ARG;
    if (n_chunks == 0) return GS2_OK;
    k_chunk_scale<<<(unsigned)n_chunks, 256, 0, (cudaStream_t)stream>>>(records, chunk_n, out);
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError() == cudaSuccess ? GS2_OK : GS2_ERR_CUDA;
}

extern "C" gs2_status gs2_mlp_grad(const uint16_t *w_bf16, const float *records, int64_t chunk_n, const int64_t *idx,
                                   int64_t nrec, const float *chunk_scale, float *partial, double *stats,
                                   gs2_stream stream) {
    if (!w_bf16 || !records || !partial || !stats || nrec < 0 || chunk_n < 1) return GS2_ERR_ARG;
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    const size_t smem = grad_smem_bytes();
    std::call_once(attr_once, [&] {
        attr_err = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (attr_err != cudaSuccess) return GS2_ERR_CUDA;
    k_mlp_grad<<<GS2_MLP_GRID, GT, smem, (cudaStream_t)stream>>>((const __nv_bfloat16 *)w_bf16, records, chunk_n,
                                                                 idx, nrec, chunk_scale, partial, stats);
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError() == cudaSuccess ? GS2_OK : GS2_ERR_CUDA;
}

extern "C" gs2_status gs2_mlp_adam(float *master, uint16_t *w_bf16, const float *partial, const double *stats,
                                   float *m, float *v, int32_t step, float lr, float beta1, float beta2, float eps,
                                   gs2_stream stream) {
    if (!master || !w_bf16 || !partial || !stats || !m || !v || step < 1) return GS2_ERR_ARG;
    k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        master, (__nv_bfloat16 *)w_bf16, partial, GS2_MLP_GRID, stats, m, v, step, lr, beta1, beta2, eps);
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError() == cudaSuccess ? GS2_OK : GS2_ERR_CUDA;
}
