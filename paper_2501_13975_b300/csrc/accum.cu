// gs2_accum_newton_blocks (Eq. local_hessian_gradient, full Newton).
//
// Pass 1 (k_accum, one CTA per screen tile, one thread per two pixels, or four
// for the position payload): walk the
// tile's depth-sorted list back to front (the order that yields the colour
// behind each Gaussian, C_back, and its transmittance T_k = T_after/(1-alpha)).
// For pixel c = C_front + T_k (alpha_k c~_k + (1 - alpha_k) C_back):
//   dc/dalpha = T_k (c~ - C_back) =: a,  dc/dc~ = alpha T_k =: w,
//   d2c/dalpha2 = 0, d2c/dalpha dc~ = T_k,
// and alpha = sigma G(z), z = (pi_x, pi_y, Sxx, Sxy, Syy).  Each pixel forms
// the group's image-space payload, the warp sums it with shuffles and the
// lanes add it with atomics into a per-view, per-Gaussian buffer zbuf[P][n]
// (L2-resident at the working-set sizes).  Every z-derivative of G is G times
// a polynomial of degree <= 4 in u = Sigma^-1 d (d the pixel offset) whose
// coefficients are the conic's, constant per Gaussian, so the geometric
// payloads are moments sum_p W u_x^i u_y^j of the per-pixel weights
// W1 = A_h alpha^2 (the Gauss-Newton part), W2 = E_a alpha (gradient and
// e-weighted curvature) and, for position, alpha times the colour-path weights:
// position 48 floats (W1 x 12 monomials, W2 x 15, cross 3 x 5, colour 6),
// scale/rotation 13 (W1 x 5, W2 x 8), opacity 2, colour 6.  The epilogue
// rebuilds the z-space gradient and Hessian from the moments and the conic
// (pos_moments_to_z, sigma_moments_to_z): about a third less arithmetic per
// (pixel, Gaussian) than forming the 20 (position) or 9 derivative terms per
// pixel, in the same number of padded reduction slots.
//
// Pass 2 (k_epi_*, one thread per Gaussian): chain rule from z to the group's
// parameters with the per-view constant Jacobians (dz/dp, d2z/dp2, dc~/dp,
// d2c~/dp2, dSigma/ds, dSigma/dtheta), added into the group's blocks; the
// zbuf entries are cleared for the next view.
#include "common.cuh"
#include "sh.cuh"

template <int G> struct Payload;
// P: accumulator floats per Gaussian and view; MIN_CTAS: resident CTAs per SM
// the register allocation is held to (65536 / (MIN_CTAS x 128) registers a thread)
template <> struct Payload<GS2_POS> { static constexpr int P = GS2_ZPOS, MIN_CTAS = 4; };
template <> struct Payload<GS2_ROT> { static constexpr int P = 13, MIN_CTAS = 7; };
template <> struct Payload<GS2_SCALE> { static constexpr int P = 13, MIN_CTAS = 7; };
template <> struct Payload<GS2_OPACITY> { static constexpr int P = 2, MIN_CTAS = 8; };
template <> struct Payload<GS2_COLOR> { static constexpr int P = 6, MIN_CTAS = 8; };

// packed upper-triangle index of a 5x5 / 3x3 symmetric matrix
__host__ __device__ constexpr int ut5(int i, int j) { return i * 5 - i * (i - 1) / 2 + (j - i); }
__host__ __device__ constexpr int ut3(int i, int j) { return i * 3 - i * (i - 1) / 2 + (j - i); }

// Moments of the geometric payloads and their conversion to the z-space sums.
// With A = Sigma^-1 = [[a, b], [b, c]] and u = A d (d = pixel - pi), the
// derivatives of G w.r.t. z = (pi_x, pi_y, S_xx, S_xy, S_yy) (S_xy counted once),
// divided by G, are
//   dG/dz = (u_x, u_y, u_x^2/2, u_x u_y, u_y^2/2) =: gz,
//   d2G/dz_i dz_j = gz_i gz_j - (the terms of A), e.g. (pi_x, pi_x): u_x^2 - a,
//   (S_xx, S_xx): u_x^4/4 - a u_x^2, (S_xy, S_xy): u_x^2 u_y^2 - a u_y^2 - 2 b u_x u_y - c u_x^2
// (see the conversions below for every entry).  The image-space sums
//   g_z = sum W2 gz,  H_zz = sum W1 gz gz^T + W2 d2G/dz2 (W2 terms left out
//   for Gauss-Newton),  cross_c = sum X_c gz
// are therefore linear in the moments of W1, W2, X_c over monomials of u.
// Monomial order of the W1 list: xx xy yy xxx xxy xyy yyy x4 x3y x2y2 xy3 y4
// (x = u_x, y = u_y); the W2 list prepends 1, x, y.
enum { MXX, MXY, MYY, MXXX, MXXY, MXYY, MYYY, MX4, MX3Y, MX2Y2, MXY3, MY4 };

// position: m[48] = W1 [12] | W2 [15] | X_c [3][5] (x, y, xx, xy, yy) | colour [6]
// -> z[41] = g_z [5] | H_zz [15] (upper, ut5) | cross [3][5] | colour [6]
__device__ __forceinline__ void pos_moments_to_z(const float (&m)[GS2_ZPOS], float a, float b, float c, bool gn,
                                                 float (&z)[GS2_ZSUM]) {
    const float *M1 = m, *M2 = m + 15;   // M2[i] = W2 moment of W1-list monomial i
    const float w0 = m[12], wx = m[13], wy = m[14];
    z[0] = wx;
    z[1] = wy;
    z[2] = 0.5f * M2[MXX];
    z[3] = M2[MXY];
    z[4] = 0.5f * M2[MYY];
    float H[15];
    H[0] = M1[MXX];                  // (0,0)
    H[1] = M1[MXY];                  // (0,1)
    H[2] = 0.5f * M1[MXXX];          // (0,2)
    H[3] = M1[MXXY];                 // (0,3)
    H[4] = 0.5f * M1[MXYY];          // (0,4)
    H[5] = M1[MYY];                  // (1,1)
    H[6] = 0.5f * M1[MXXY];          // (1,2)
    H[7] = M1[MXYY];                 // (1,3)
    H[8] = 0.5f * M1[MYYY];          // (1,4)
    H[9] = 0.25f * M1[MX4];          // (2,2)
    H[10] = 0.5f * M1[MX3Y];         // (2,3)
    H[11] = 0.25f * M1[MX2Y2];       // (2,4)
    H[12] = M1[MX2Y2];               // (3,3)
    H[13] = 0.5f * M1[MXY3];         // (3,4)
    H[14] = 0.25f * M1[MY4];         // (4,4)
    if (!gn) {
        H[0] += M2[MXX] - a * w0;
        H[1] += M2[MXY] - b * w0;
        H[2] += 0.5f * M2[MXXX] - a * wx;
        H[3] += M2[MXXY] - a * wy - b * wx;
        H[4] += 0.5f * M2[MXYY] - b * wy;
        H[5] += M2[MYY] - c * w0;
        H[6] += 0.5f * M2[MXXY] - b * wx;
        H[7] += M2[MXYY] - b * wy - c * wx;
        H[8] += 0.5f * M2[MYYY] - c * wy;
        H[9] += 0.25f * M2[MX4] - a * M2[MXX];
        H[10] += 0.5f * M2[MX3Y] - a * M2[MXY] - b * M2[MXX];
        H[11] += 0.25f * M2[MX2Y2] - b * M2[MXY];
        H[12] += M2[MX2Y2] - a * M2[MYY] - 2.f * b * M2[MXY] - c * M2[MXX];
        H[13] += 0.5f * M2[MXY3] - b * M2[MYY] - c * M2[MXY];
        H[14] += 0.25f * M2[MY4] - c * M2[MYY];
    }
#pragma unroll
    for (int i = 0; i < 15; ++i) z[5 + i] = H[i];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float *X = m + 27 + 5 * ch;
        z[20 + 5 * ch + 0] = X[0];
        z[20 + 5 * ch + 1] = X[1];
        z[20 + 5 * ch + 2] = 0.5f * X[2];
        z[20 + 5 * ch + 3] = X[3];
        z[20 + 5 * ch + 4] = 0.5f * X[4];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) z[35 + i] = m[42 + i];
}

// scaling / rotation: m[13] = W1 [x4 x3y x2y2 xy3 y4] | W2 [xx xy yy x4 x3y x2y2 xy3 y4]
// -> z[9] = g over (S_xx, S_xy, S_yy) [3] | H [6] (upper, ut3)
__device__ __forceinline__ void sigma_moments_to_z(const float (&m)[13], float a, float b, float c, bool gn,
                                                   float (&z)[9]) {
    z[0] = 0.5f * m[5];
    z[1] = m[6];
    z[2] = 0.5f * m[7];
    z[3] = 0.25f * m[0];
    z[4] = 0.5f * m[1];
    z[5] = 0.25f * m[2];
    z[6] = m[2];
    z[7] = 0.5f * m[3];
    z[8] = 0.25f * m[4];
    if (!gn) {
        z[3] += 0.25f * m[8] - a * m[5];
        z[4] += 0.5f * m[9] - a * m[6] - b * m[5];
        z[5] += 0.25f * m[10] - b * m[6];
        z[6] += m[10] - a * m[7] - 2.f * b * m[6] - c * m[5];
        z[7] += 0.5f * m[11] - b * m[7] - c * m[6];
        z[8] += 0.25f * m[12] - c * m[7];
    }
}

// Warp sum of a P-float payload followed by atomic adds into zbuf[i][k].
// Reduce-scatter transpose: the payload is padded to PP = 2^m floats; at each
// butterfly step a lane keeps half of its current values (chosen by its lane
// bit) and adds the partner's matching half, so after the five steps lane L
// holds fully reduced entries at distinct indices (PP/32 of them when PP >= 32,
// or one entry shared by 32/PP lanes).  P (5 - 1/32) shuffles become about PP,
// and the atomics are issued by many lanes at once instead of lane 0 alone.
// A payload longer than 32 is reduced in two parts, the first 32 entries and
// the rest (41 = 32 + 9 -> 32 + 16 padded slots instead of 64).
template <int P> struct Pad { static constexpr int PP = P <= 2 ? 2 : P <= 4 ? 4 : P <= 8 ? 8 : P <= 16 ? 16 : P <= 32 ? 32 : 64; };

// TOP: first butterfly offset; 16 reduces over the whole warp, 8 over each
// half-warp separately (one step fewer, twice the atomics -- measured slower
// for the position payload on the scene workload, so 16 is used)
// STORE (deterministic mode): instead of the atomics, every reduced entry
// (zeros included) is stored to row[OFF + idx] (shared memory).
template <int Q, int OFF, int P, typename ACC, int TOP = 16, bool STORE = false>
__device__ __forceinline__ void reduce_scatter_part(const float (&pl)[P], int lane, ACC *__restrict__ zbuf, int n,
                                                    uint32_t k, float *row = nullptr) {
    constexpr int PP = Pad<Q>::PP;
    constexpr int GROUP_LANES = 2 * TOP;   // lanes that end up sharing one reduction
    float v[PP];
#pragma unroll
    for (int i = 0; i < PP; ++i) v[i] = (i < Q) ? pl[OFF + i] : 0.f;
    int off = 0;           // index of v[0] in this part
    int len = PP;          // values this lane still holds
#pragma unroll
    for (int o = TOP; o > 0; o >>= 1) {
        const bool up = (lane & o) != 0;
        if (len > 1) {
            const int h = len >> 1;
#pragma unroll
            for (int i = 0; i < PP / 2; ++i) {
                if (i < h) {
                    const float send = up ? v[i] : v[i + h];
                    const float keep = up ? v[i + h] : v[i];
                    v[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, o);
                }
            }
            if (up) off += h;
            len = h;
        } else {
            v[0] += __shfl_xor_sync(0xFFFFFFFFu, v[0], o);
        }
    }
    // lanes that share an entry (PP < GROUP_LANES): only the one with the low lane bits clear writes
    constexpr int share = (PP >= GROUP_LANES) ? 1 : GROUP_LANES / PP;
    if ((lane & (share - 1)) == 0) {
#pragma unroll
        for (int j = 0; j < (PP >= GROUP_LANES ? PP / GROUP_LANES : 1); ++j) {
            const int idx = off + j;
            if constexpr (STORE) {
                if (idx < Q) row[OFF + idx] = v[j];
            } else {
                if (idx < Q && v[j] != 0.f) atomicAdd(&zbuf[(size_t)(OFF + idx) * n + k], (ACC)v[j]);
            }
        }
    }
}

template <int P, typename ACC>
__device__ __forceinline__ void warp_reduce_scatter_add(const float (&pl)[P], int lane, ACC *__restrict__ zbuf,
                                                        int n, uint32_t k) {
    if constexpr (P > 32) {
        reduce_scatter_part<32, 0, P, ACC>(pl, lane, zbuf, n, k);
        reduce_scatter_part<P - 32, 32, P, ACC>(pl, lane, zbuf, n, k);
    } else {
        reduce_scatter_part<P, 0, P, ACC>(pl, lane, zbuf, n, k);
    }
}

// The warp sum of the payload stored to row[0 .. P) (deterministic mode).
template <int P>
__device__ __forceinline__ void warp_reduce_scatter_store(const float (&pl)[P], int lane, float *row) {
    if constexpr (P > 32) {
        reduce_scatter_part<32, 0, P, float, 16, true>(pl, lane, nullptr, 0, 0u, row);
        reduce_scatter_part<P - 32, 32, P, float, 16, true>(pl, lane, nullptr, 0, 0u, row);
    } else {
        reduce_scatter_part<P, 0, P, float, 16, true>(pl, lane, nullptr, 0, 0u, row);
    }
}

// Deterministic mode: list entries per flush of the per-warp sums
#define GS2_DET_CHUNK 32

// Packed FP32 pairs: the sm_100-family f32x2 instructions (add, mul, fma on a
// 64-bit register pair, each half rounded as its scalar _rn counterpart) do the
// same operation for both pixels of a lane in one issue slot.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// back-to-front state of the two pixels of a lane (x: q = 0, y: q = 1)
struct PairState {
    float2 T, cb0, cb1, cb2;
};

// One list entry for the pixel pair of a lane, branch free: a pixel that does
// not composite the Gaussian (outside the image, past its last contributor,
// or outside the support) takes alpha = 0 and keeps its state, and the
// payload weight ap (alpha where composited and not clamped, else 0) zeroes
// the falloff terms of clamped and inactive pixels.  The payload is kept per
// pixel (pl[i].x, pl[i].y) and summed before the warp reduction.
// e, h: (q = 0, q = 1) pairs of the pixels' loss derivatives per channel.
template <int GROUP, int P>
__device__ __forceinline__ void pair_payload(PairState &ps, const float2 (&e)[3], const float2 (&h)[3],
                                             const float4 &A, const float4 &B, const float4 &C, float2 G,
                                             float2 al, float2 ap, bool l0, bool l1, float dx, float2 dy,
                                             float2 (&pl)[P]) {
    const float2 om = fma2(al, f2(-1.f), f2(1.f));   // 1 - alpha, rounded once
    float2 Tk = mul2(ps.T, make_float2(rcp_approx(om.x), rcp_approx(om.y)));
    Tk.x = l0 ? Tk.x : ps.T.x;
    Tk.y = l1 ? Tk.y : ps.T.y;
    const float2 w = mul2(al, Tk);
    if constexpr (GROUP == GS2_COLOR) {
        const float2 ww = mul2(w, w);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            pl[c] = fma2(w, e[c], pl[c]);
            pl[3 + c] = fma2(ww, h[c], pl[3 + c]);
        }
    } else {
        const float2 a0 = mul2(Tk, fma2(ps.cb0, f2(-1.f), f2(C.x)));
        const float2 a1 = mul2(Tk, fma2(ps.cb1, f2(-1.f), f2(C.y)));
        const float2 a2 = mul2(Tk, fma2(ps.cb2, f2(-1.f), f2(C.z)));
        const float2 Ea = fma2(e[2], a2, fma2(e[1], a1, mul2(e[0], a0)));
        const float2 Ah = fma2(mul2(h[2], a2), a2, fma2(mul2(h[1], a1), a1, mul2(mul2(h[0], a0), a0)));
        if constexpr (GROUP == GS2_OPACITY) {
            const float2 Gp = make_float2(ap.x != 0.f ? G.x : 0.f, ap.y != 0.f ? G.y : 0.f);
            pl[0] = fma2(Ea, Gp, pl[0]);
            pl[1] = fma2(mul2(Ah, Gp), Gp, pl[1]);
        } else {   // rotation / scaling: moments over (x4 x3y x2y2 xy3 y4) and (xx xy yy x4 ... y4)
            const float2 dxv = f2(dx);
            const float2 ux = fma2(f2(A.z), dxv, mul2(f2(A.w), dy));
            const float2 uy = fma2(f2(A.w), dxv, mul2(f2(B.x), dy));
            const float2 xx = mul2(ux, ux), xy = mul2(ux, uy), yy = mul2(uy, uy);
            const float2 m4[5] = {mul2(xx, xx), mul2(xx, xy), mul2(xx, yy), mul2(xy, yy), mul2(yy, yy)};
            const float2 W1 = mul2(mul2(Ah, ap), ap), W2 = mul2(Ea, ap);
#pragma unroll
            for (int i = 0; i < 5; ++i) pl[i] = fma2(W1, m4[i], pl[i]);
            pl[5] = fma2(W2, xx, pl[5]);
            pl[6] = fma2(W2, xy, pl[6]);
            pl[7] = fma2(W2, yy, pl[7]);
#pragma unroll
            for (int i = 0; i < 5; ++i) pl[8 + i] = fma2(W2, m4[i], pl[8 + i]);
        }
        ps.cb0 = fma2(al, f2(C.x), mul2(om, ps.cb0));
        ps.cb1 = fma2(al, f2(C.y), mul2(om, ps.cb1));
        ps.cb2 = fma2(al, f2(C.z), mul2(om, ps.cb2));
    }
    ps.T = Tk;
}

// The position payload of one list entry for the NPR pixel pairs of a lane
// (NPR = 1: two pixels, 2: four), straight into the 48 moment slots: each
// moment is the f32x2 sum over the pairs of weight x monomial, then the two
// halves added.  Colour and cross terms first, so that e, h and the colour-
// path weights die before the 27 geometric moments are formed.
// gn (Gauss-Newton): the e-weighted second derivatives of the pixel colour
// (e d2c/dz2 through the falloff, e d2c/dalpha dc~) are left out.
// hi(pl) is called once slots 32..47 (two of the cross-term channels and the
// colour sums) are formed, lo(pl) once slots 0..31 are: the warp reduction of
// the first part runs before the second part's moments exist, so fewer of the
// 48 slots are live at once.
template <int NPR, typename Hi, typename Lo>
__device__ __forceinline__ void pos_pairs(PairState (&ps)[NPR], const float2 (&e)[NPR][3],
                                          const float2 (&h)[NPR][3], const float4 &A, const float4 &B,
                                          const float4 &C, const float2 (&al)[NPR], const float2 (&ap)[NPR],
                                          const bool (&lv)[NPR][2], float dx, const float2 (&dy)[NPR], bool gn,
                                          float (&pl)[GS2_ZPOS], Hi &&hi, Lo &&lo) {
    float2 W1[NPR], W2[NPR], X[NPR][3], UX[NPR], UY[NPR];
    float2 sc[6];   // colour sums: w e_c, w^2 h_c
    const float2 dxv = f2(dx);
#pragma unroll
    for (int r = 0; r < NPR; ++r) {
        const float2 om = fma2(al[r], f2(-1.f), f2(1.f));   // 1 - alpha, rounded once
        float2 Tk = mul2(ps[r].T, make_float2(rcp_approx(om.x), rcp_approx(om.y)));
        Tk.x = lv[r][0] ? Tk.x : ps[r].T.x;
        Tk.y = lv[r][1] ? Tk.y : ps[r].T.y;
        const float2 w = mul2(al[r], Tk), ww = mul2(w, w);
        const float2 a0 = mul2(Tk, fma2(ps[r].cb0, f2(-1.f), f2(C.x)));
        const float2 a1 = mul2(Tk, fma2(ps[r].cb1, f2(-1.f), f2(C.y)));
        const float2 a2 = mul2(Tk, fma2(ps[r].cb2, f2(-1.f), f2(C.z)));
        const float2 ac[3] = {a0, a1, a2};
        const float2 Ea = fma2(e[r][2], a2, fma2(e[r][1], a1, mul2(e[r][0], a0)));
        const float2 Ah = fma2(mul2(h[r][2], a2), a2, fma2(mul2(h[r][1], a1), a1, mul2(mul2(h[r][0], a0), a0)));
        W1[r] = mul2(mul2(Ah, ap[r]), ap[r]);
        W2[r] = mul2(Ea, ap[r]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 et = gn ? f2(0.f) : mul2(e[r][c], Tk);
            X[r][c] = mul2(fma2(mul2(h[r][c], ac[c]), w, et), ap[r]);
            sc[c] = r == 0 ? mul2(w, e[r][c]) : fma2(w, e[r][c], sc[c]);
            sc[3 + c] = r == 0 ? mul2(ww, h[r][c]) : fma2(ww, h[r][c], sc[3 + c]);
        }
        UX[r] = fma2(f2(A.z), dxv, mul2(f2(A.w), dy[r]));
        UY[r] = fma2(f2(A.w), dxv, mul2(f2(B.x), dy[r]));
        ps[r].cb0 = fma2(al[r], f2(C.x), mul2(om, ps[r].cb0));
        ps[r].cb1 = fma2(al[r], f2(C.y), mul2(om, ps[r].cb1));
        ps[r].cb2 = fma2(al[r], f2(C.z), mul2(om, ps[r].cb2));
        ps[r].T = Tk;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) pl[42 + i] = sc[i].x + sc[i].y;
    // sum over the pairs of wt[r] m[r], both halves added
    auto msum = [](const float2 (&wt)[NPR], const float2 (&m)[NPR]) {
        float2 s = mul2(wt[0], m[0]);
#pragma unroll
        for (int r = 1; r < NPR; ++r) s = fma2(wt[r], m[r], s);
        return s.x + s.y;
    };
    float2 XX[NPR], XY[NPR], YY[NPR];
#pragma unroll
    for (int r = 0; r < NPR; ++r) {
        XX[r] = mul2(UX[r], UX[r]);
        XY[r] = mul2(UX[r], UY[r]);
        YY[r] = mul2(UY[r], UY[r]);
    }
    auto cross = [&](int c) {   // cross terms: X_c over (x, y, xx, xy, yy)
        float2 Xc[NPR];
#pragma unroll
        for (int r = 0; r < NPR; ++r) Xc[r] = X[r][c];
        pl[27 + 5 * c + 0] = msum(Xc, UX);
        pl[27 + 5 * c + 1] = msum(Xc, UY);
        pl[27 + 5 * c + 2] = msum(Xc, XX);
        pl[27 + 5 * c + 3] = msum(Xc, XY);
        pl[27 + 5 * c + 4] = msum(Xc, YY);
    };
    cross(1);
    cross(2);
    hi(pl);   // slots 32..47
    cross(0);
    {
        float2 s = W2[0];
#pragma unroll
        for (int r = 1; r < NPR; ++r) s = add2(W2[r], s);
        pl[12] = s.x + s.y;
    }
    pl[13] = msum(W2, UX);
    pl[14] = msum(W2, UY);
    // monomials in the W1-list order: xx xy yy xxx xxy xyy yyy x4 x3y x2y2 xy3 y4
    auto both = [&](int i, const float2 (&m)[NPR]) {
        pl[i] = msum(W1, m);
        pl[15 + i] = msum(W2, m);
    };
    both(MXX, XX);
    both(MXY, XY);
    both(MYY, YY);
    float2 m[NPR];
#pragma unroll
    for (int r = 0; r < NPR; ++r) m[r] = mul2(XX[r], UX[r]);
    both(MXXX, m);
#pragma unroll
    for (int r = 0; r < NPR; ++r) m[r] = mul2(XX[r], UY[r]);
    both(MXXY, m);
#pragma unroll
    for (int r = 0; r < NPR; ++r) m[r] = mul2(XY[r], UY[r]);
    both(MXYY, m);
#pragma unroll
    for (int r = 0; r < NPR; ++r) m[r] = mul2(YY[r], UY[r]);
    both(MYYY, m);
#pragma unroll
    for (int r = 0; r < NPR; ++r) m[r] = mul2(XX[r], XX[r]);
    both(MX4, m);
#pragma unroll
    for (int r = 0; r < NPR; ++r) m[r] = mul2(XX[r], XY[r]);
    both(MX3Y, m);
#pragma unroll
    for (int r = 0; r < NPR; ++r) m[r] = mul2(XX[r], YY[r]);
    both(MX2Y2, m);
#pragma unroll
    for (int r = 0; r < NPR; ++r) m[r] = mul2(XY[r], YY[r]);
    both(MXY3, m);
#pragma unroll
    for (int r = 0; r < NPR; ++r) m[r] = mul2(YY[r], YY[r]);
    both(MY4, m);
    lo(pl);   // slots 0..31
}

// DET (deterministic mode): no atomics.  Every list entry's payload is the
// sum of the tile's four warp sums taken in warp order, written to
// det_part[sorted position][P] (entries past the tile's last contributor
// get zero rows); k_det_reduce then sums each Gaussian's entries in a fixed
// order into zbuf.
// NQ: pixels per thread (2, or 4 for the position payload, whose warp
// reduction costs about as much as the payload itself: four pixels a lane
// pay it once per 128 pixels).  NQ = 2: NT threads, warp w
// covers an 8x8 block, lane l the pixels (l % 8, l / 8 + 4 q); NQ = 4: two
// warps per 16x16 tile, each an 8-wide column of the tile, lane l the pixels
// (l % 8, l / 8 + 4 q), q = 0..3.
template <int GROUP, int NQ> struct AccumShape {
    static constexpr int NT = GS2_TILE_PIX / NQ;   // threads per tile
    static constexpr int NW = NT / 32;
    static constexpr int MIN_CTAS = NQ == 2 ? Payload<GROUP>::MIN_CTAS : GROUP == GS2_POS ? 8 : 12;
    // four pixels a thread: e and h of the pixels in shared memory (24 registers
    // fewer) and half-size staging batches, so that 8 CTAs (16 warps) fit on an SM
    static constexpr bool EH_SMEM = NQ == 4;
    static constexpr int NB = EH_SMEM ? GS2_TILE_PIX / 2 : GS2_TILE_PIX;   // list entries staged per batch
    static_assert(NT % 32 == 0, "a tile holds whole warps");
};

// SPLIT: a persistent grid takes work items (tile, [c0, c1), checkpoint slot)
// from `items` through the fetch counter ctrl[1] (ctrl[0] items), so that one
// long tile walk is shared by several CTAs.  A pixel whose last contributor
// lies behind c1 starts from the compositing's checkpoint at c1: T(c1), and
// the colour behind, (colour its entries from c1 on add) / T(c1); the others
// from the final state, as the whole walk does.
template <int GROUP, typename ACC, bool DET = false, int NQ = 2, bool SPLIT = false>
__global__ void __launch_bounds__(AccumShape<GROUP, NQ>::NT, AccumShape<GROUP, NQ>::MIN_CTAS) k_accum(const uint2 *__restrict__ ranges,
                                                           const uint32_t *__restrict__ ids, ProjView pv,
                                                           RasterView rv, const float *__restrict__ E,
                                                           const float *__restrict__ Hh, int W, int H, int tiles_x,
                                                           float amin, float amax, int gn, ACC *__restrict__ zbuf,
                                                           int n, unsigned long long *__restrict__ active_stat,
                                                           float *__restrict__ det_part,
                                                           const uint32_t *__restrict__ tile_order,
                                                           const uint4 *__restrict__ items,
                                                           uint32_t *__restrict__ ctrl) {
    constexpr int P = Payload<GROUP>::P;
    constexpr int NT = AccumShape<GROUP, NQ>::NT, NW = AccumShape<GROUP, NQ>::NW;
    constexpr bool EH_SMEM = AccumShape<GROUP, NQ>::EH_SMEM;
    constexpr int NB = AccumShape<GROUP, NQ>::NB;     // list entries staged per batch
    constexpr int NPR = NQ / 2;                       // pixel pairs a thread (f32x2 arithmetic)
    static_assert(NQ == 2 || (NQ == 4 && GS2_TILE == 16), "four pixels a thread need 16x16 tiles");
    static_assert(!(DET && SPLIT), "the deterministic mode walks whole tiles");
    constexpr int PER = NB / NT;                      // entries each thread stages
    // two staging buffers: batch b + 1 is copied in while batch b is walked
    __shared__ uint32_t sId[2][NB];
    __shared__ float4 sA[2][NB], sB[2][NB], sC[2][NB];
    __shared__ uint32_t sMax;
    __shared__ uint4 sItem;
    // four pixels a thread: e, h of pixel pair r of thread t as f32x2 pairs,
    // [r][0] = (e0, e1), [r][1] = (e2, h0), [r][2] = (h1, h2) (each .x: q = 2r, .y: q = 2r + 1)
    __shared__ float4 sEP[EH_SMEM ? NPR : 1][3][EH_SMEM ? NT : 1];
    __shared__ float sDet[DET ? NW : 1][DET ? GS2_DET_CHUNK : 1][DET ? P : 1];   // per-warp sums of a chunk
    const int t = threadIdx.x, lane = t & 31;
    if constexpr (DET) {
        for (int q = t; q < NW * GS2_DET_CHUNK * P; q += NT) (&sDet[0][0][0])[q] = 0.f;
    }
    const int wb = t >> 5;   // warp block: (wb % GS2_WPR) 8 columns, (wb / GS2_WPR) 4 NQ rows
    const size_t PI = (size_t)W * H;
    uint32_t nact = 0u;   // (pixel, Gaussian) evaluations this thread did (profile statistic)
    for (;;) {
        int tile, c0 = 0, c1 = 0x7FFFFFFF;   // list entries [c0, c1) of the tile's walk
        uint32_t slot = 0xFFFFFFFFu;        // checkpoint at c1
        if constexpr (SPLIT) {
            if (t == 0) {
                const uint32_t i = atomicAdd(&ctrl[1], 1u);
                sItem = i < ctrl[0] ? items[i] : make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
            }
            __syncthreads();
            const uint4 w = sItem;
            if (w.x == 0xFFFFFFFFu) break;   // CTA-uniform
            tile = (int)w.x;
            c0 = (int)w.y;
            c1 = (int)w.z;
            slot = w.w;
        } else {
            tile = tile_order ? (int)tile_order[blockIdx.x] : (int)blockIdx.x;   // longest lists first
        }
        const int tcol = tile % tiles_x, trow = tile / tiles_x;
        const int lx = (wb % GS2_WPR) * 8 + (t & 7), ly0 = (wb / GS2_WPR) * (4 * NQ) + ((t >> 3) & 3);
        const int px = tcol * GS2_TILE + lx;
        const int py = trow * GS2_TILE + ly0;
        uint32_t last[NQ];
        PairState pst[NPR];
        float2 pe2[EH_SMEM ? 1 : NPR][3], ph2[EH_SMEM ? 1 : NPR][3];   // e, h in registers (two pixels a thread)
        float2 pyf[NPR];
#pragma unroll
        for (int r = 0; r < NPR; ++r) {
            float e[2][3], h[2][3], T[2], cb[2][3];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int y = py + 4 * (2 * r + j);
                const bool inside = px < W && y < H;
                last[2 * r + j] = 0u;   // outside the image: no list entry is composited
                T[j] = 1.f;
#pragma unroll
                for (int c = 0; c < 3; ++c) e[j][c] = h[j][c] = cb[j][c] = 0.f;
                if (inside) {
                    const size_t pp = (size_t)y * W + px;
                    last[2 * r + j] = rv.last[pp];
                    T[j] = rv.tfinal[pp];
                    if constexpr (SPLIT) {
                        if (last[2 * r + j] > (uint32_t)c1) {   // composites past c1: start at the checkpoint
                            const int lp = (ly0 + 4 * (2 * r + j)) * GS2_TILE + lx;
                            const float4 ck = rv.ck[(size_t)slot * GS2_TILE_PIX + lp];
                            T[j] = ck.x;
                            // T >= t_min > 0 where the compositing went on; with t_min = 0 an
                            // underflowed T leaves every weight in front zero, as the whole walk does
                            const float iT = ck.x > 0.f ? 1.f / ck.x : 0.f;
                            cb[j][0] = ck.y * iT;
                            cb[j][1] = ck.z * iT;
                            cb[j][2] = ck.w * iT;
                        }
                    }
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        e[j][c] = E[c * PI + pp];
                        h[j][c] = Hh[c * PI + pp];
                    }
                }
            }
            pst[r].T = make_float2(T[0], T[1]);
            pst[r].cb0 = make_float2(cb[0][0], cb[1][0]);
            pst[r].cb1 = make_float2(cb[0][1], cb[1][1]);
            pst[r].cb2 = make_float2(cb[0][2], cb[1][2]);
            pyf[r] = make_float2((float)(py + 8 * r), (float)(py + 8 * r + 4));
            if constexpr (EH_SMEM) {
                sEP[r][0][t] = make_float4(e[0][0], e[1][0], e[0][1], e[1][1]);
                sEP[r][1][t] = make_float4(e[0][2], e[1][2], h[0][0], h[1][0]);
                sEP[r][2][t] = make_float4(h[0][1], h[1][1], h[0][2], h[1][2]);
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    pe2[r][c] = make_float2(e[0][c], e[1][c]);
                    ph2[r][c] = make_float2(h[0][c], h[1][c]);
                }
            }
        }
        uint32_t last2 = last[0];
#pragma unroll
        for (int q = 1; q < NQ; ++q) last2 = max(last2, last[q]);
        if (t == 0) sMax = 0u;
        __syncthreads();
        atomicMax(&sMax, last2);
        __syncthreads();
        const int maxlast = (int)sMax;
        const int hi = min(c1, maxlast);   // end of this walk
        // this warp's own end of list: its lanes have nothing to do beyond it
        const int wlast = (int)__reduce_max_sync(0xFFFFFFFFu, last2);
        const uint2 r = ranges[tile];
        const float fx = (float)px;
        // batches back to front: batch b covers [max(c0, hi - NB (b + 1)), hi - NB b)
        const int nbat = hi > c0 ? (hi - c0 + NB - 1) / NB : 0;
        auto list_index = [&](int b, int i) { return hi - NB * (b + 1) + t + i * NT; };
        uint32_t knext[PER];
        auto fetch = [&](int b) {
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int li = list_index(b, i);
                knext[i] = li >= c0 ? ids[r.x + li] : 0u;
            }
        };
        auto issue = [&](int b) {
            const int buf = b & 1;
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int j = t + i * NT;
                if (list_index(b, i) >= c0) {
                    const uint32_t k = knext[i];
                    sId[buf][j] = k;
                    cp_async16(&sA[buf][j], &pv.recA[k]);
                    cp_async16(&sB[buf][j], &pv.recB[k]);
                    if constexpr (GROUP != GS2_COLOR) cp_async16(&sC[buf][j], &pv.col[k]);   // colour: no c~
                }
            }
            cp_async_commit();
        };
        if (nbat > 0) {
            fetch(0);
            issue(0);
            if (nbat > 1) fetch(1);
        }
        for (int b = 0; b < nbat; ++b) {
            cp_async_wait_all();
            __syncthreads();   // batch b visible to all; everyone is done with batch b - 1's buffer
            if (b + 1 < nbat) {
                issue(b + 1);
                if (b + 2 < nbat) fetch(b + 2);
            }
            const int buf = b & 1;
            const int bend = hi - NB * b, bbeg = max(c0, bend - NB);
            const int base = bend - NB;   // list index of slot 0 of this batch (may be negative)
            // one list entry (back to front): its payload, then the warp sum
            // (atomics, or stored to `row` in deterministic mode)
            auto entry = [&](int jj, float *row) {
                const int s = jj - base;
                const float4 A = sA[buf][s], B = sB[buf][s];
                const float dx = __fsub_rn(fx, A.x);
                const float2 dxv = f2(dx);
                float2 dy[NPR], qf[NPR];
                bool lv[NPR][2];
                bool any = false;
#pragma unroll
                for (int r = 0; r < NPR; ++r) {
                    dy[r] = add2(pyf[r], f2(-A.y));
                    // dec_quad of both pixels (the same correctly rounded operations, in the same order)
                    float2 qa = fma2(f2(A.z), dxv, mul2(f2(A.w), dy[r]));
                    qa = fma2(f2(A.w), dy[r], qa);
                    qf[r] = fma2(dxv, qa, mul2(mul2(f2(B.x), dy[r]), dy[r]));
                    lv[r][0] = (uint32_t)jj < last[2 * r] && qf[r].x <= B.z;   // composited (as k_raster)
                    lv[r][1] = (uint32_t)jj < last[2 * r + 1] && qf[r].y <= B.z;
                    any = any || lv[r][0] || lv[r][1];
                    nact += (lv[r][0] ? 1u : 0u) + (lv[r][1] ? 1u : 0u);
                }
                if (!__any_sync(0xFFFFFFFFu, any)) return;
                float2 G[NPR], al[NPR], ap[NPR];
#pragma unroll
                for (int r = 0; r < NPR; ++r) {
                    const float2 xg = mul2(qf[r], f2(-0.72134752044448170368f));   // gs2_falloff, both pixels
                    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(G[r].x) : "f"(xg.x));
                    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(G[r].y) : "f"(xg.y));
                    const bool c0 = qf[r].x < B.w, c1 = qf[r].y < B.w;   // clamped at alpha_max
                    al[r] = mul2(f2(B.y), G[r]);
                    al[r].x = lv[r][0] ? (c0 ? amax : al[r].x) : 0.f;
                    al[r].y = lv[r][1] ? (c1 ? amax : al[r].y) : 0.f;
                    ap[r] = make_float2(c0 ? 0.f : al[r].x, c1 ? 0.f : al[r].y);
                }
                float4 C = make_float4(0.f, 0.f, 0.f, 0.f);
                if constexpr (GROUP != GS2_COLOR) C = sC[buf][s];
                float pl[P];
                if constexpr (GROUP == GS2_POS) {
                    float2 pe[NPR][3], ph[NPR][3];
#pragma unroll
                    for (int r = 0; r < NPR; ++r) {
                        if constexpr (EH_SMEM) {
                            const float4 k0 = sEP[r][0][t], k1 = sEP[r][1][t], k2 = sEP[r][2][t];
                            pe[r][0] = make_float2(k0.x, k0.y);
                            pe[r][1] = make_float2(k0.z, k0.w);
                            pe[r][2] = make_float2(k1.x, k1.y);
                            ph[r][0] = make_float2(k1.z, k1.w);
                            ph[r][1] = make_float2(k2.x, k2.y);
                            ph[r][2] = make_float2(k2.z, k2.w);
                        } else {
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                pe[r][c] = pe2[r][c];
                                ph[r][c] = ph2[r][c];
                            }
                        }
                    }
                    const uint32_t k = sId[buf][s];
                    pos_pairs<NPR>(
                        pst, pe, ph, A, B, C, al, ap, lv, dx, dy, gn != 0, pl,
                        [&](const float (&v)[P]) {
                            if constexpr (DET)
                                reduce_scatter_part<P - 32, 32, P, float, 16, true>(v, lane, nullptr, 0, 0u, row);
                            else
                                reduce_scatter_part<P - 32, 32, P, ACC>(v, lane, zbuf, n, k);
                        },
                        [&](const float (&v)[P]) {
                            if constexpr (DET)
                                reduce_scatter_part<32, 0, P, float, 16, true>(v, lane, nullptr, 0, 0u, row);
                            else
                                reduce_scatter_part<32, 0, P, ACC>(v, lane, zbuf, n, k);
                        });
                    return;
                } else {
                    float2 pl2[P];
#pragma unroll
                    for (int i = 0; i < P; ++i) pl2[i] = f2(0.f);
#pragma unroll
                    for (int r = 0; r < NPR; ++r) {
                        if constexpr (EH_SMEM) {
                            const float4 k0 = sEP[r][0][t], k1 = sEP[r][1][t], k2 = sEP[r][2][t];
                            const float2 pe[3] = {make_float2(k0.x, k0.y), make_float2(k0.z, k0.w), make_float2(k1.x, k1.y)};
                            const float2 ph[3] = {make_float2(k1.z, k1.w), make_float2(k2.x, k2.y), make_float2(k2.z, k2.w)};
                            pair_payload<GROUP, P>(pst[r], pe, ph, A, B, C, G[r], al[r], ap[r], lv[r][0], lv[r][1], dx,
                                                   dy[r], pl2);
                        } else {
                            pair_payload<GROUP, P>(pst[r], pe2[r], ph2[r], A, B, C, G[r], al[r], ap[r], lv[r][0],
                                                   lv[r][1], dx, dy[r], pl2);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < P; ++i) pl[i] = pl2[i].x + pl2[i].y;
                }
                if constexpr (DET)
                    warp_reduce_scatter_store<P>(pl, lane, row);
                else
                    warp_reduce_scatter_add<P, ACC>(pl, lane, zbuf, n, sId[buf][s]);
            };
            if constexpr (DET) {
                const int w = t >> 5;
                for (int c1 = bend; c1 > bbeg; c1 -= GS2_DET_CHUNK) {   // CTA-uniform chunks
                    const int c0 = max(bbeg, c1 - GS2_DET_CHUNK);
                    for (int jj = min(c1, wlast) - 1; jj >= c0; --jj) entry(jj, &sDet[w][jj - c0][0]);
                    __syncthreads();
                    const int cnt = (c1 - c0) * P;
                    for (int q = t; q < cnt; q += NT) {
                        const int e = q / P, i = q - e * P;
                        float v = sDet[0][e][i];
                        sDet[0][e][i] = 0.f;
#pragma unroll
                        for (int ww = 1; ww < NW; ++ww) {   // warp order
                            v = __fadd_rn(v, sDet[ww][e][i]);
                            sDet[ww][e][i] = 0.f;
                        }
                        det_part[(size_t)(r.x + (uint32_t)(c0 + e)) * P + i] = v;
                    }
                    __syncthreads();
                }
            } else {
                for (int jj = min(bend, wlast) - 1; jj >= bbeg; --jj) entry(jj, nullptr);
            }
        }
        if constexpr (DET) {   // entries past the last contributor of every pixel contribute nothing
            const int nl = (int)(r.y - r.x);
            for (int q = t + maxlast * P; q < nl * P; q += NT) det_part[(size_t)r.x * P + q] = 0.f;
        }
        if constexpr (!SPLIT) break;
        __syncthreads();   // this item's shared memory is free before the next item is fetched
    }
    if (active_stat) {
        unsigned long long c = nact;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
        if (lane == 0 && c) atomicAdd(active_stat, c);
    }
}

// ------------------------------------------------------------------ epilogues
struct GaussGeo {
    float p[3], s[3], R[3][3];
};

__device__ __forceinline__ void load_geo(const DevScene &sc, int k, GaussGeo &g) {
    const int n = sc.n;
    for (int i = 0; i < 3; ++i) {
        g.p[i] = sc.mean[i * n + k];
        g.s[i] = sc.scale[i * n + k];
    }
    float qw = sc.quat[k], qx = sc.quat[n + k], qy = sc.quat[2 * n + k], qz = sc.quat[3 * n + k];
    const float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw *= qn; qx *= qn; qy *= qn; qz *= qn;
    g.R[0][0] = 1.f - 2.f * (qy * qy + qz * qz); g.R[0][1] = 2.f * (qx * qy - qw * qz); g.R[0][2] = 2.f * (qx * qz + qw * qy);
    g.R[1][0] = 2.f * (qx * qy + qw * qz); g.R[1][1] = 1.f - 2.f * (qx * qx + qz * qz); g.R[1][2] = 2.f * (qy * qz - qw * qx);
    g.R[2][0] = 2.f * (qx * qz - qw * qy); g.R[2][1] = 2.f * (qy * qz + qw * qx); g.R[2][2] = 1.f - 2.f * (qx * qx + qy * qy);
}

// camera-space centre and the 2x3 T = J Wr
__device__ __forceinline__ void cam_T(const DevCam &cam, const float p[3], float t[3], float T[2][3]) {
    const float *V = cam.V;
    for (int i = 0; i < 3; ++i) t[i] = V[i * 4] * p[0] + V[i * 4 + 1] * p[1] + V[i * 4 + 2] * p[2] + V[i * 4 + 3];
    const float iz = 1.f / t[2];
    const float taux = fminf(fmaxf(t[0] * iz, -cam.Lx), cam.Lx), tauy = fminf(fmaxf(t[1] * iz, -cam.Ly), cam.Ly);
    const float j00 = cam.fx * iz, j02 = -cam.fx * taux * iz, j11 = cam.fy * iz, j12 = -cam.fy * tauy * iz;
    for (int j = 0; j < 3; ++j) {
        T[0][j] = j00 * V[j] + j02 * V[8 + j];
        T[1][j] = j11 * V[4 + j] + j12 * V[8 + j];
    }
}

// S2 = T S3 T^T as the parameter vector (xx, xy, yy)
__device__ __forceinline__ void push_cov(const float T[2][3], const float S3[3][3], float out[3]) {
    float TS[2][3];
    for (int a = 0; a < 2; ++a)
        for (int j = 0; j < 3; ++j) TS[a][j] = T[a][0] * S3[0][j] + T[a][1] * S3[1][j] + T[a][2] * S3[2][j];
    out[0] = TS[0][0] * T[0][0] + TS[0][1] * T[0][1] + TS[0][2] * T[0][2];
    out[1] = TS[0][0] * T[1][0] + TS[0][1] * T[1][1] + TS[0][2] * T[1][2];
    out[2] = TS[1][0] * T[1][0] + TS[1][1] * T[1][1] + TS[1][2] * T[1][2];
}

template <typename ACC>
__global__ void k_epi_opacity(const ProjView pv, ACC *__restrict__ zbuf, int n, float *__restrict__ blocks) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || pv.touched[k] == 0u) return;
    const float z0 = (float)zbuf[k], z1 = (float)zbuf[n + k];
    atomicAdd(&blocks[k], z0);          // the views of a group may run concurrently
    atomicAdd(&blocks[n + k], z1);
    zbuf[k] = 0.f;
    zbuf[n + k] = 0.f;
}

template <typename ACC>
__global__ void k_epi_color(DevScene sc, DevCam cam, const ProjView pv, ACC *zbuf, float *slot) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = sc.n;
    if (k >= n) return;
    const bool vis = pv.touched[k] != 0u;
    float zz[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) zz[i] = vis ? (float)zbuf[(size_t)i * n + k] : 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i) slot[(size_t)i * n + k] = zz[i];
    if (vis)
#pragma unroll
        for (int i = 0; i < 6; ++i) zbuf[(size_t)i * n + k] = 0.f;
    float rx = sc.mean[k] - cam.o[0], ry = sc.mean[n + k] - cam.o[1], rz = sc.mean[2 * n + k] - cam.o[2];
    const float rn = rsqrtf(rx * rx + ry * ry + rz * rz);
    float phi[GS2_MAX_SH];
    sh_phi(sc.S, rx * rn, ry * rn, rz * rn, phi);
    for (int i = 0; i < sc.S; ++i) slot[(size_t)(6 + i) * n + k] = sh_norm(i) * phi[i];
}

// gn (Gauss-Newton) in the epilogues: the terms g_z . d2z/dy2 (the
// image-space gradient times the second derivatives of the projected
// quantities) are left out.
template <typename ACC>
__global__ void k_epi_scale(DevScene sc, DevCam cam, const ProjView pv, ACC *__restrict__ zbuf,
                            float *__restrict__ blocks, int gn) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = sc.n;
    if (k >= n || pv.touched[k] == 0u) return;
    // every load first (accumulators, the block entries updated, parameters):
    // they are then in flight together instead of one memory latency each
    float mo[13], z[9];
#pragma unroll
    for (int i = 0; i < 13; ++i) mo[i] = (float)zbuf[(size_t)i * n + k];
    const float4 cA = pv.recA[k], cB = pv.recB[k];   // conic (a, b) and c
    GaussGeo g;
    load_geo(sc, k, g);
#pragma unroll
    for (int i = 0; i < 13; ++i) zbuf[(size_t)i * n + k] = 0.f;
    sigma_moments_to_z(mo, cA.z, cA.w, cB.x, gn != 0, z);
    float t[3], T[2][3];
    cam_T(cam, g.p, t, T);
    float dS[3][3], d2S[3][3];  // [param j][(xx,xy,yy)]
    for (int j = 0; j < 3; ++j) {
        const float m0 = T[0][0] * g.R[0][j] + T[0][1] * g.R[1][j] + T[0][2] * g.R[2][j];
        const float m1 = T[1][0] * g.R[0][j] + T[1][1] * g.R[1][j] + T[1][2] * g.R[2][j];
        d2S[j][0] = 2.f * m0 * m0; d2S[j][1] = 2.f * m0 * m1; d2S[j][2] = 2.f * m1 * m1;
        for (int a = 0; a < 3; ++a) dS[j][a] = g.s[j] * d2S[j][a];
    }
    float Hz[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b) Hz[a][b] = Hz[b][a] = z[3 + ut3(a, b)];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float gj = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) gj += z[a] * dS[j][a];
        atomicAdd(&blocks[(size_t)j * n + k], gj);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int l = j; l < 3; ++l) {
            float hv = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) hv += dS[j][a] * Hz[a][b] * dS[l][b];
            if (j == l && !gn)
#pragma unroll
                for (int a = 0; a < 3; ++a) hv += z[a] * d2S[j][a];
            atomicAdd(&blocks[(size_t)(3 + ut3(j, l)) * n + k], hv);
        }
}

template <typename ACC>
__global__ void k_epi_rot(DevScene sc, DevCam cam, DevCam primary, const ProjView pv, ACC *__restrict__ zbuf,
                          float *__restrict__ blocks, int gn) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = sc.n;
    if (k >= n || pv.touched[k] == 0u) return;
    float mo[13], z[9];
#pragma unroll
    for (int i = 0; i < 13; ++i) mo[i] = (float)zbuf[(size_t)i * n + k];
    const float4 cA = pv.recA[k], cB = pv.recB[k];   // conic (a, b) and c
    GaussGeo g;
    load_geo(sc, k, g);
#pragma unroll
    for (int i = 0; i < 13; ++i) zbuf[(size_t)i * n + k] = 0.f;
    sigma_moments_to_z(mo, cA.z, cA.w, cB.x, gn != 0, z);
    float t[3], T[2][3];
    cam_T(cam, g.p, t, T);
    // Sigma3 = R diag(s^2) R^T; K = [a]x with a the primary view direction
    float S3[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            float acc = 0.f;
            for (int l = 0; l < 3; ++l) acc += g.R[i][l] * g.s[l] * g.s[l] * g.R[j][l];
            S3[i][j] = acc;
        }
    float a[3] = {g.p[0] - primary.o[0], g.p[1] - primary.o[1], g.p[2] - primary.o[2]};
    const float an = rsqrtf(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    for (int i = 0; i < 3; ++i) a[i] *= an;
    const float K[3][3] = {{0.f, -a[2], a[1]}, {a[2], 0.f, -a[0]}, {-a[1], a[0], 0.f}};
    float KS[3][3], SK[3][3], KSK[3][3], K2S[3][3], SK2[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            float ks = 0.f, sk = 0.f;
            for (int l = 0; l < 3; ++l) {
                ks += K[i][l] * S3[l][j];
                sk += S3[i][l] * K[l][j];
            }
            KS[i][j] = ks;
            SK[i][j] = sk;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            float ksk = 0.f, k2s = 0.f, sk2 = 0.f;
            for (int l = 0; l < 3; ++l) {
                ksk += KS[i][l] * K[l][j];
                k2s += K[i][l] * KS[l][j];
                sk2 += SK[i][l] * K[l][j];
            }
            KSK[i][j] = ksk;
            K2S[i][j] = k2s;
            SK2[i][j] = sk2;
        }
    float D1[3][3], D2[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            D1[i][j] = KS[i][j] - SK[i][j];
            D2[i][j] = K2S[i][j] - 2.f * KSK[i][j] + SK2[i][j];
        }
    float d1[3], d2[3];
    push_cov(T, D1, d1);
    push_cov(T, D2, d2);
    float gth = 0.f, hth = 0.f;
    for (int aa = 0; aa < 3; ++aa) {
        gth += z[aa] * d1[aa];
        if (!gn) hth += z[aa] * d2[aa];
        for (int b = 0; b < 3; ++b) {
            const float hz = z[3 + (aa <= b ? ut3(aa, b) : ut3(b, aa))];
            hth += d1[aa] * hz * d1[b];
        }
    }
    atomicAdd(&blocks[k], gth);
    atomicAdd(&blocks[n + k], hth);
}

// Position epilogue.  With u = 1/t_z and a, b in {x, y}:
//   pi_a = f_a t_a u + c_a,
//   Sigma_ab = f_a f_b u^2 Q_ab(tau) (+ low-pass), tau_a = clamp(t_a u),
// V the camera-space 3D covariance (J V J^T written out); derivatives by the
// chain rule through the intermediates (u, tau_x, tau_y).
template <typename ACC, int S>
__global__ void __launch_bounds__(128, 6) k_epi_pos(DevScene sc, DevCam cam, const ProjView pv,
                                                    ACC *__restrict__ zbuf, float *__restrict__ blocks, int gn) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = sc.n;
    if (k >= n || pv.touched[k] == 0u) return;
    float z[GS2_ZSUM];
    {
        float mo[GS2_ZPOS];
        // all loads first, then the clears (interleaving them serialises the loads)
#pragma unroll
        for (int i = 0; i < GS2_ZPOS; ++i) mo[i] = (float)zbuf[(size_t)i * n + k];
        const float4 cA = pv.recA[k], cB = pv.recB[k];   // conic (a, b) and c
#pragma unroll
        for (int i = 0; i < GS2_ZPOS; ++i) zbuf[(size_t)i * n + k] = 0.f;
        pos_moments_to_z(mo, cA.z, cA.w, cB.x, gn != 0, z);
    }
    GaussGeo g;
    load_geo(sc, k, g);
    const float *V = cam.V;
    float t[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) t[i] = V[i * 4] * g.p[0] + V[i * 4 + 1] * g.p[1] + V[i * 4 + 2] * g.p[2] + V[i * 4 + 3];
    const float u = 1.f / t[2], u2 = u * u, u3 = u2 * u;
    // camera-space covariance Vc = (Wr R diag(s)) (Wr R diag(s))^T
    float M3[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            M3[i][j] = (V[i * 4] * g.R[0][j] + V[i * 4 + 1] * g.R[1][j] + V[i * 4 + 2] * g.R[2][j]) * g.s[j];
    float Vc[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Vc[i][j] = M3[i][0] * M3[j][0] + M3[i][1] * M3[j][1] + M3[i][2] * M3[j][2];
    const float f[2] = {cam.fx, cam.fy};
    // dz[i][k]: derivative of z_i w.r.t. t_k; Gt = sum_i z_i d2z_i/dt2 (symmetric 3x3)
    float dz[5][3];
    float Gt[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) Gt[a][b] = 0.f;
#pragma unroll
    for (int a = 0; a < 2; ++a) {      // pi_a
        dz[a][0] = (a == 0) ? f[0] * u : 0.f;
        dz[a][1] = (a == 1) ? f[1] * u : 0.f;
        dz[a][2] = -f[a] * t[a] * u2;
        Gt[a][2] += -f[a] * u2 * z[a];
        Gt[2][a] += -f[a] * u2 * z[a];
        Gt[2][2] += 2.f * f[a] * t[a] * u3 * z[a];
    }
    // Sigma_ab = f_a f_b u^2 Q_ab(tau), Q_ab = V_ab - tau_a V_zb - tau_b V_za + tau_a tau_b V_zz,
    // tau_a = t_a u clamped to the frustum limit (constant where clamped).
    // Intermediates y = (u, tau_x, tau_y): Jacobian Jy[m][k] = dy_m/dt_k, Hessians Hy[m].
    const float Lc[2] = {cam.Lx, cam.Ly};
    float tau[2];
    bool cl[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float tr = t[a] * u;
        cl[a] = fabsf(tr) > Lc[a];
        tau[a] = fminf(fmaxf(tr, -Lc[a]), Lc[a]);
    }
    float Jy[3][3], Hy[3][3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Jy[m][a] = 0.f;
#pragma unroll
            for (int b = 0; b < 3; ++b) Hy[m][a][b] = 0.f;
        }
    Jy[0][2] = -u2;
    Hy[0][2][2] = 2.f * u3;
#pragma unroll
    for (int a = 0; a < 2; ++a)
        if (!cl[a]) {
            Jy[1 + a][a] = u;
            Jy[1 + a][2] = -t[a] * u2;
            Hy[1 + a][a][2] = -u2;
            Hy[1 + a][2][a] = -u2;
            Hy[1 + a][2][2] = 2.f * t[a] * u3;
        }
    const int EA[3] = {0, 0, 1}, EB[3] = {0, 1, 1};
#pragma unroll
    for (int e = 0; e < 3; ++e) {      // Sigma_ab
        const int a = EA[e], b = EB[e];
        const float ff = f[a] * f[b];
        const float Vab = Vc[a][b], Vzb = Vc[2][b], Vza = Vc[2][a], Vzz = Vc[2][2];
        const float Q = Vab - tau[a] * Vzb - tau[b] * Vza + tau[a] * tau[b] * Vzz;
        float dQ[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float dac = (a == c) ? 1.f : 0.f, dbc = (b == c) ? 1.f : 0.f;
            dQ[c] = -dac * Vzb - dbc * Vza + (dac * tau[b] + dbc * tau[a]) * Vzz;
        }
        float Fy[3], Fyy[3][3];
        Fy[0] = 2.f * ff * u * Q;
        Fy[1] = ff * u2 * dQ[0];
        Fy[2] = ff * u2 * dQ[1];
        Fyy[0][0] = 2.f * ff * Q;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            Fyy[0][1 + c] = Fyy[1 + c][0] = 2.f * ff * u * dQ[c];
#pragma unroll
            for (int d = 0; d < 2; ++d)
                Fyy[1 + c][1 + d] =
                    ff * u2 * (((a == c) && (b == d) ? 1.f : 0.f) + ((b == c) && (a == d) ? 1.f : 0.f)) * Vzz;
        }
        const float ze = z[2 + e];
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) dz[2 + e][kk] = Fy[0] * Jy[0][kk] + Fy[1] * Jy[1][kk] + Fy[2] * Jy[2][kk];
        float FJ[3][3];   // Fyy Jy
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) FJ[m][kk] = Fyy[m][0] * Jy[0][kk] + Fyy[m][1] * Jy[1][kk] + Fyy[m][2] * Jy[2][kk];
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < 3; ++k2) {
                const float sec = Jy[0][k1] * FJ[0][k2] + Jy[1][k1] * FJ[1][k2] + Jy[2][k1] * FJ[2][k2] +
                                  Fy[0] * Hy[0][k1][k2] + Fy[1] * Hy[1][k1][k2] + Fy[2] * Hy[2][k1][k2];
                Gt[k1][k2] += ze * sec;
            }
    }
    // to world coordinates: Jzp = dz Wr, sum_i z_i d2z_i/dp2 = Wr^T Gt Wr
    float Jzp[5][3];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c) Jzp[i][c] = dz[i][0] * V[c] + dz[i][1] * V[4 + c] + dz[i][2] * V[8 + c];
    float gp[3], Hp[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < 5; ++i) acc += Jzp[i][c] * z[i];
        gp[c] = acc;
    }
    float HJ[5][3];   // Hzz Jzp
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j < 5; ++j) acc += z[5 + (i <= j ? ut5(i, j) : ut5(j, i))] * Jzp[j][c];
            HJ[i][c] = acc;
        }
    float GW[3][3];   // Gt Wr
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int d = 0; d < 3; ++d) GW[a][d] = Gt[a][0] * V[d] + Gt[a][1] * V[4 + d] + Gt[a][2] * V[8 + d];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = c; d < 3; ++d) {
            float acc = 0.f;
#pragma unroll
            for (int i = 0; i < 5; ++i) acc += Jzp[i][c] * HJ[i][d];
            if (!gn)
#pragma unroll
                for (int a = 0; a < 3; ++a) acc += V[a * 4 + c] * GW[a][d];
            Hp[c][d] = acc;
        }
    // colour path: c~(p) through r(p)
    float r[3] = {g.p[0] - cam.o[0], g.p[1] - cam.o[1], g.p[2] - cam.o[2]};
    const float rho = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]), irho = 1.f / rho;
#pragma unroll
    for (int i = 0; i < 3; ++i) r[i] *= irho;
    float Pm[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) Pm[a][b] = ((a == b ? 1.f : 0.f) - r[a] * r[b]) * irho;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float WE = z[35 + ch], SS = z[38 + ch];
        float wco[S];   // unrolled: the S loads of a channel are in flight together
#pragma unroll
        for (int i = 0; i < S; ++i) wco[i] = sh_norm(i) * __ldcs(sc.sh + (size_t)(ch * S + i) * n + k);
        float fv, gr[3], hs[6];
        sh_poly_derivs(S, wco, r[0], r[1], r[2], fv, gr, hs);
        const float Hr[3][3] = {{hs[0], hs[1], hs[2]}, {hs[1], hs[3], hs[4]}, {hs[2], hs[4], hs[5]}};
        float gc[3], y[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) gc[a] = Pm[a][0] * gr[0] + Pm[a][1] * gr[1] + Pm[a][2] * gr[2];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float acc = 0.f;
#pragma unroll
            for (int i = 0; i < 5; ++i) acc += Jzp[i][c] * z[20 + ch * 5 + i];
            y[c] = acc;
        }
        float HPm[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) HPm[a][b] = Hr[a][0] * Pm[0][b] + Hr[a][1] * Pm[1][b] + Hr[a][2] * Pm[2][b];
        const float gdr = gr[0] * r[0] + gr[1] * r[1] + gr[2] * r[2];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gp[a] += WE * gc[a];
#pragma unroll
            for (int b = a; b < 3; ++b) {
                float h2 = Pm[a][0] * HPm[0][b] + Pm[a][1] * HPm[1][b] + Pm[a][2] * HPm[2][b];
                // sum_m gr_m d2r_m/dp_a dp_b = (3 (gr.r) r_a r_b - gr_a r_b - gr_b r_a - d_ab (gr.r)) / rho^2
                h2 += (3.f * gdr * r[a] * r[b] - gr[a] * r[b] - gr[b] * r[a] - (a == b ? gdr : 0.f)) * irho * irho;
                Hp[a][b] += y[a] * gc[b] + gc[a] * y[b] + SS * gc[a] * gc[b] + (gn ? 0.f : WE * h2);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) atomicAdd(&blocks[(size_t)c * n + k], gp[c]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b) atomicAdd(&blocks[(size_t)(3 + ut3(a, b)) * n + k], Hp[a][b]);
}

// Deterministic mode: each Gaussian's image-space payload is the sum of its
// list entries' partials (det_part rows) taken in emission order (the tiles of
// its rectangle row by row), written to zbuf[P][n] for the epilogues.  FP32
// sums are compensated (Kahan: the rounding error of every addition is carried
// into the next); with mixed precision (ACC = double) the sum is FP64.  One
// warp per depth rank r (Gaussian order[r]), lane i summing payload entry i
// (and i + 32), so every partial row is read by one coalesced access; emitted
// pairs past the pair capacity and box tiles the support ellipse misses
// (dropped by the tile sort: ids_emit = 0xFFFFFFFF) hold no entry and are skipped.
template <int P, typename ACC>
__global__ void __launch_bounds__(128) k_det_reduce(const uint32_t *__restrict__ order, const uint32_t *__restrict__ offs,
                                                    const uint32_t *__restrict__ tsort, int n,
                                                    const uint32_t *__restrict__ count,
                                                    const uint32_t *__restrict__ inv,
                                                    const uint32_t *__restrict__ ids_emit,
                                                    const float *__restrict__ part, ACC *__restrict__ zbuf) {
    constexpr int NE = (P + 31) / 32;   // entries per lane
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= n) return;
    const uint32_t cnt = tsort[r];
    if (cnt == 0u) return;
    const uint32_t id = order[r], M = count[0];
    const uint32_t j0 = offs[r], j1 = min(j0 + cnt, M);
    ACC acc[NE];
    float comp[NE];
#pragma unroll
    for (int e = 0; e < NE; ++e) {
        acc[e] = 0;
        comp[e] = 0.f;
    }
    for (uint32_t j = j0; j < j1; ++j) {
        if (ids_emit[j] == 0xFFFFFFFFu) continue;   // dropped pair
        const uint32_t sp = inv[j];
        const float *row = part + (size_t)sp * P;
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            const int i = lane + 32 * e;
            if (i < P) {
                const float v = row[i];
                if constexpr (sizeof(ACC) == sizeof(float)) {
                    const float y = __fsub_rn(v, comp[e]);
                    const float t = __fadd_rn((float)acc[e], y);
                    comp[e] = __fsub_rn(__fsub_rn(t, (float)acc[e]), y);
                    acc[e] = t;
                } else {
                    acc[e] += (ACC)v;
                }
            }
        }
    }
#pragma unroll
    for (int e = 0; e < NE; ++e) {
        const int i = lane + 32 * e;
        if (i < P) zbuf[(size_t)i * n + id] = acc[e];
    }
}

// Work items of the split accumulation: every tile's walk [0, maxlast) cut at
// multiples of ca, in the tiles' launch order (longest lists first), the back
// item of a tile first; an item ending below the walk's end names the
// checkpoint slot at its end.  One CTA: per-thread runs of tiles, a block scan
// of their item counts, then the items written in order.  Also resets the
// fetch counter of the persistent accumulation grid.
__global__ void __launch_bounds__(1024) k_accum_items(const uint32_t *__restrict__ order,
                                                      const uint32_t *__restrict__ maxlast,
                                                      const uint2 *__restrict__ ranges, int ntiles, int ca,
                                                      uint4 *__restrict__ items, uint32_t *__restrict__ ctrl) {
    __shared__ uint32_t wsum[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int per = (ntiles + 1023) / 1024;
    const int i0 = min(ntiles, t * per), i1 = min(ntiles, i0 + per);
    const uint32_t uca = (uint32_t)ca;
    uint32_t cnt = 0u;
    for (int i = i0; i < i1; ++i) cnt += (maxlast[order ? (int)order[i] : i] + uca - 1u) / uca;
    uint32_t inc = cnt;   // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        const uint32_t v = wsum[lane];
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        wsum[lane] = x - v;
        if (lane == 31) {
            ctrl[0] = x;
            ctrl[1] = 0u;
        }
    }
    __syncthreads();
    uint32_t pos = wsum[w] + inc - cnt;
    for (int i = i0; i < i1; ++i) {
        const int tile = order ? (int)order[i] : i;
        const uint32_t np = (maxlast[tile] + uca - 1u) / uca, base = ranges[tile].x / uca;
        for (uint32_t s = np; s-- > 0u;)
            items[pos++] = make_uint4((uint32_t)tile, s * uca, (s + 1u) * uca, s + 1u == np ? 0xFFFFFFFFu : base + s + 1u);
    }
}

static int device_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    return sms;
}

struct AccumArgs {
    const uint2 *ranges;
    const uint32_t *ids;
    ProjView pv;
    RasterView rv;
    const float *E, *Hh;
    int W, H, tiles_x;
    float amin, amax;
    int gn, n;
    unsigned long long *act;
    const uint32_t *tile_order;
    const uint4 *items;
    uint32_t *ctrl;
    dim3 grid;
};

// resident CTAs per SM of a split accumulation kernel (first asked for by
// prepare_split_kernels, from the host, outside any stream capture)
template <int G, typename ACC, int NQ>
static int split_occupancy() {
    static int occ = 0;
    if (!occ) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_accum<G, ACC, false, NQ, true>,
                                                      AccumShape<G, NQ>::NT, 0);
        if (occ < 1) occ = 1;
    }
    return occ;
}

void prepare_split_kernels() {
    device_sms();
#define GS2_SPLIT_PREP(ACC)                                                                                      \
    split_occupancy<GS2_POS, ACC, 2>();                                                                          \
    split_occupancy<GS2_ROT, ACC, 2>();                                                                          \
    split_occupancy<GS2_SCALE, ACC, 2>();                                                                        \
    split_occupancy<GS2_OPACITY, ACC, 2>();                                                                      \
    split_occupancy<GS2_COLOR, ACC, 2>();
    GS2_SPLIT_PREP(float)
    GS2_SPLIT_PREP(double)
#undef GS2_SPLIT_PREP
#if GS2_TILE == 16
    split_occupancy<GS2_POS, float, 4>();
    split_occupancy<GS2_COLOR, float, 4>();
    split_occupancy<GS2_POS, double, 4>();
    split_occupancy<GS2_COLOR, double, 4>();
#endif
}

// one accumulation launch (atomics, not the deterministic mode): a CTA per tile, or
// (split) a persistent grid of as many CTAs as are resident at once
template <int G, typename ACC, int NQ>
static void accum_launch(const AccumArgs &a, ACC *zb, bool split, cudaStream_t st) {
    constexpr int NT = AccumShape<G, NQ>::NT;
    if (split) {
        const int occ = split_occupancy<G, ACC, NQ>();
        k_accum<G, ACC, false, NQ, true><<<(unsigned)(device_sms() * occ), NT, 0, st>>>(
            a.ranges, a.ids, a.pv, a.rv, a.E, a.Hh, a.W, a.H, a.tiles_x, a.amin, a.amax, a.gn, zb, a.n, a.act,
            (float *)nullptr, nullptr, a.items, a.ctrl);
    } else {
        k_accum<G, ACC, false, NQ, false><<<a.grid, NT, 0, st>>>(a.ranges, a.ids, a.pv, a.rv, a.E, a.Hh, a.W, a.H,
                                                                 a.tiles_x, a.amin, a.amax, a.gn, zb, a.n, a.act,
                                                                 (float *)nullptr, a.tile_order, nullptr, nullptr);
    }
}

template <typename ACC>
static void launch_accum_t(gs2_ctx *ctx, int group, const DevScene &sc, const DevCam &view, const DevCam &primary,
                           ProjView pv, RasterView rv, const gs2_config &cfg, int view_slot, void *blocks, dim3 grid,
                           const uint32_t *ids, bool prof, cudaStream_t st) {
    const int n = sc.n;
    ACC *zb = (ACC *)ctx->zbuf;
    gs2_ctx *pc = ctx->owner ? ctx->owner : ctx;   // profile pool and statistics
    unsigned long long *act = pc->prof_on ? pc->d_stats + 5 * group + 3 : nullptr;
    const bool det = cfg.deterministic != 0 && ctx->det_part && ctx->det_order;
    // split walks: the last compositing on this context kept its checkpoints
    const bool split = !det && ctx->rs_split > 0 && ctx->ck && ctx->acc_items;
    if (split) {
        rv.ck = ctx->ck;
        rv.ck_every = ctx->rs_split;
        k_accum_items<<<1, 1024, 0, st>>>(ctx->tile_order, ctx->tile_maxlast, ctx->ranges, (int)grid.x,
                                          ctx->rs_split, ctx->acc_items, ctx->acc_ctrl);
        GS2_COUNT_LAUNCH(1);
    }
    const AccumArgs a = {ctx->ranges, ids, pv, rv, ctx->pix_e, ctx->pix_h, view.w, view.h, ctx->tiles_x,
                         cfg.alpha_min, cfg.alpha_max, cfg.gauss_newton, n, act, ctx->tile_order, ctx->acc_items,
                         ctx->acc_ctrl, grid};
#define ACC_LAUNCH(G)                                                                                             \
    do {                                                                                                          \
        if (det) {                                                                                                \
            k_accum<G, float, true><<<grid, GS2_PAIR_THREADS, 0, st>>>(                                           \
                ctx->ranges, ids, pv, rv, ctx->pix_e, ctx->pix_h, view.w, view.h, ctx->tiles_x, cfg.alpha_min,    \
                cfg.alpha_max, cfg.gauss_newton, (float *)nullptr, n, act, ctx->det_part, ctx->tile_order,        \
                nullptr, nullptr);                                                                                \
            if (n > 0)                                                                                            \
                k_det_reduce<Payload<G>::P, ACC><<<(n + 3) / 4, 128, 0, st>>>(                                    \
                    ctx->det_order, pv.offs, pv.tsort, n, ctx->d_count, ctx->det_inv, ctx->det_ids,               \
                    ctx->det_part, zb);                                                                           \
        } else {                                                                                                  \
            accum_launch<G, ACC, 2>(a, zb, split, st);                                                            \
        }                                                                                                         \
    } while (0)
#if GS2_TILE == 16
    // four pixels per thread (position, colour): two warps per tile
#define ACC_LAUNCH4(G)                                                                                           \
    if (!det && ctx->accum_px == 4) {                                                                            \
        accum_launch<G, ACC, 4>(a, zb, split, st);                                                               \
        break;                                                                                                   \
    }
#else
#define ACC_LAUNCH4(G)
#endif
    switch (group) {
    case GS2_POS: ACC_LAUNCH4(GS2_POS) ACC_LAUNCH(GS2_POS); break;
    // measured per sweep (two / four pixels a thread): rotation and scaling
    // 1.30 / 1.34 ms, opacity 0.85 / 0.89, colour 0.75 / 0.71
    case GS2_ROT: ACC_LAUNCH(GS2_ROT); break;
    case GS2_SCALE: ACC_LAUNCH(GS2_SCALE); break;
    case GS2_OPACITY: ACC_LAUNCH(GS2_OPACITY); break;
    default: ACC_LAUNCH4(GS2_COLOR) ACC_LAUNCH(GS2_COLOR); break;
    }
#undef ACC_LAUNCH4
#undef ACC_LAUNCH
    if (det) GS2_COUNT_LAUNCH(1);
    if (prof) {
        cudaEventRecord(pc->prof_ev[2 * pc->prof_n + 1], st);
        pc->prof_n++;
    }
    GS2_COUNT_LAUNCH(2);
    if (n == 0) return;
    const int eg = (n + 255) / 256;
    const int gn = cfg.gauss_newton;
    float *b = (float *)blocks;
    switch (group) {
    case GS2_POS:
        switch (sc.S) {
        case 1: k_epi_pos<ACC, 1><<<(n + 127) / 128, 128, 0, st>>>(sc, view, pv, zb, b, gn); break;
        case 4: k_epi_pos<ACC, 4><<<(n + 127) / 128, 128, 0, st>>>(sc, view, pv, zb, b, gn); break;
        case 9: k_epi_pos<ACC, 9><<<(n + 127) / 128, 128, 0, st>>>(sc, view, pv, zb, b, gn); break;
        default: k_epi_pos<ACC, 16><<<(n + 127) / 128, 128, 0, st>>>(sc, view, pv, zb, b, gn); break;
        }
        break;
    case GS2_ROT: k_epi_rot<ACC><<<eg, 256, 0, st>>>(sc, view, primary, pv, zb, b, gn); break;
    case GS2_SCALE: k_epi_scale<ACC><<<eg, 256, 0, st>>>(sc, view, pv, zb, b, gn); break;
    case GS2_OPACITY: k_epi_opacity<ACC><<<eg, 256, 0, st>>>(pv, zb, n, b); break;
    default: {
        float *slot = b + (size_t)view_slot * (6 + sc.S) * n;
        k_epi_color<ACC><<<eg, 256, 0, st>>>(sc, view, pv, zb, slot);
    }
    }
}

cudaError_t launch_accum(gs2_ctx *ctx, int group, const DevScene &sc, const DevCam &view, const DevCam &primary,
                         ProjView pv, RasterView rv, const gs2_config &cfg, int view_slot, void *blocks,
                         cudaStream_t st) {
    dim3 grid((unsigned)(ctx->tiles_x * ctx->tiles_y));
    const uint32_t *ids = ctx->list_ids;
    gs2_ctx *pc = ctx->owner ? ctx->owner : ctx;   // profile pool (shared by a sweep's view lanes)
    const bool prof = pc->prof_on && pc->prof_n < GS2_PROF_POOL;
    if (prof) {
        cudaEventRecord(pc->prof_ev[2 * pc->prof_n], st);
        pc->prof_group[pc->prof_n] = group;
    }
    if (cfg.precision == 0)
        launch_accum_t<float>(ctx, group, sc, view, primary, pv, rv, cfg, view_slot, blocks, grid, ids, prof, st);
    else
        launch_accum_t<double>(ctx, group, sc, view, primary, pv, rv, cfg, view_slot, blocks, grid, ids, prof, st);
    return cudaGetLastError();
}
