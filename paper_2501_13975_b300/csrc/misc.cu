// Small kernels around the hot path: f x f box downsampling of secondary
// targets (Sec. 4.3) and the bounding sphere of the means (Sec. 4.1).
#include "common.cuh"

__global__ void k_downsample(const float *__restrict__ in, int W, int H, int f, float *__restrict__ out) {
    const int W2 = W / f, H2 = H / f;
    const size_t P2 = (size_t)W2 * H2, P = (size_t)W * H;
    const float inv = 1.f / (float)(f * f);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < 3 * P2; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / P2);
        const size_t rem = i % P2;
        const int y = (int)(rem / W2), x = (int)(rem % W2);
        float s = 0.f;
        for (int dy = 0; dy < f; ++dy)
            for (int dx = 0; dx < f; ++dx) s += in[c * P + (size_t)(y * f + dy) * W + x * f + dx];
        out[i] = s * inv;
    }
}

cudaError_t launch_downsample(const float *in, int w, int h, int f, float *out, cudaStream_t st) {
    const size_t n = 3 * (size_t)(w / f) * (h / f);
    if (n == 0) return cudaSuccess;
    const int grid = (int)std::min<size_t>((n + 255) / 256, 148 * 16);
    k_downsample<<<grid, 256, 0, st>>>(in, w, h, f, out);
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError();
}

// one CTA: axis-aligned box of the means, then the largest distance to its centre
__global__ void __launch_bounds__(1024) k_bsphere(DevScene sc, float *out) {
    __shared__ float s[6][32];
    __shared__ float cen[3];
    const int n = sc.n, t = threadIdx.x, lane = t & 31, w = t >> 5;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int k = t; k < n; k += blockDim.x)
        for (int i = 0; i < 3; ++i) {
            const float v = sc.mean[(size_t)i * n + k];
            lo[i] = fminf(lo[i], v);
            hi[i] = fmaxf(hi[i], v);
        }
    for (int i = 0; i < 3; ++i)
        for (int o = 16; o > 0; o >>= 1) {
            lo[i] = fminf(lo[i], __shfl_xor_sync(0xFFFFFFFFu, lo[i], o));
            hi[i] = fmaxf(hi[i], __shfl_xor_sync(0xFFFFFFFFu, hi[i], o));
        }
    if (lane == 0)
        for (int i = 0; i < 3; ++i) {
            s[i][w] = lo[i];
            s[3 + i][w] = hi[i];
        }
    __syncthreads();
    if (t < 3) {
        float a = INFINITY, b = -INFINITY;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) {
            a = fminf(a, s[t][j]);
            b = fmaxf(b, s[3 + t][j]);
        }
        cen[t] = 0.5f * (a + b);
    }
    __syncthreads();
    float r2 = 0.f;
    for (int k = t; k < n; k += blockDim.x) {
        float d = 0.f;
        for (int i = 0; i < 3; ++i) {
            const float v = sc.mean[(size_t)i * n + k] - cen[i];
            d += v * v;
        }
        r2 = fmaxf(r2, d);
    }
    for (int o = 16; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xFFFFFFFFu, r2, o));
    __syncthreads();
    if (lane == 0) s[0][w] = r2;
    __syncthreads();
    if (t == 0) {
        float m = 0.f;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) m = fmaxf(m, s[0][j]);
        out[0] = cen[0];
        out[1] = cen[1];
        out[2] = cen[2];
        out[3] = sqrtf(m);
    }
}

cudaError_t launch_bounding_sphere(const DevScene &sc, float *out, cudaStream_t st) {
    k_bsphere<<<1, 1024, 0, st>>>(sc, out);
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError();
}
