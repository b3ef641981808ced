// Reproducible FP32 decisions of the forward pass (Sec. 3, Eq. 3dgs).
//
// Three discrete decisions of the path rest on floating point:
//   - which tiles list a Gaussian (its support { sigma G >= alpha_min } reaches
//     a pixel of the tile),
//   - whether a (pixel, Gaussian) term is composited (sigma G >= alpha_min),
//   - whether its alpha is clamped (sigma G > alpha_max).
// They are taken here in FP32 from the FP32 parameters with correctly rounded
// operations only (add, sub, mul, fma, div, sqrt; floor / ceil / min / max are
// exact) in a stated order, and without any library transcendental: the
// logarithm of the thresholds is the atanh (Gregory) series below.  Any IEEE
// FP32 implementation that performs the same operations in the same order
// obtains the same bits, so the decisions are reproducible outside this
// library, bit for bit.  Expressed through the quadratic form q = d^T Sigma^-1 d
// of the pixel offset d, the term decisions are
//   composited  <=>  q <= l    = 2 ln(sigma / alpha_min),
//   clamped     <=>  q <  lmax = 2 ln(sigma / alpha_max)  (lmax = -1 if sigma <= alpha_max),
// the same sets as sigma exp(-q/2) >= alpha_min and > alpha_max in exact
// arithmetic.  (The composited values -- alpha, transmittance, colour -- are
// computed separately with ordinary FP32 arithmetic.)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define D_ADD(a, b) __fadd_rn((a), (b))
#define D_SUB(a, b) __fsub_rn((a), (b))
#define D_MUL(a, b) __fmul_rn((a), (b))
#define D_FMA(a, b, c) __fmaf_rn((a), (b), (c))
#define D_DIV(a, b) __fdiv_rn((a), (b))
#define D_SQRT(a) __fsqrt_rn(a)

// Natural logarithm of a finite x >= 1.  x = 2^e m with m in [sqrt(1/2),
// sqrt(2)] (exact), ln m = 2 atanh(u) = 2 (u + u^3/3 + u^5/5 + u^7/7 + u^9/9),
// u = (m - 1)/(m + 1), |u| <= 0.172 (the next term is below 2^-27 of the sum);
// ln x = e ln 2 + ln m.  Error a few 1e-7 absolute: decisions only need the
// value to be the same everywhere, not correctly rounded.
__device__ __forceinline__ float dec_ln(float x) {
    const uint32_t b = __float_as_uint(x);
    int e = (int)((b >> 23) & 0xFFu) - 127;
    float m = __uint_as_float((b & 0x7FFFFFu) | 0x3F800000u);   // [1, 2)
    if (m > 0x1.6a09e6p+0f) {                                     // sqrt(2)
        m = D_MUL(m, 0.5f);
        e += 1;
    }
    const float u = D_DIV(D_SUB(m, 1.f), D_ADD(m, 1.f));
    const float s = D_MUL(u, u);
    float p = 0x1.c71c72p-4f;           // 1/9
    p = D_FMA(p, s, 0x1.24924ap-3f);    // 1/7
    p = D_FMA(p, s, 0x1.99999ap-3f);    // 1/5
    p = D_FMA(p, s, 0x1.555556p-2f);    // 1/3
    p = D_FMA(p, s, 1.f);
    const float lm = D_MUL(D_MUL(2.f, u), p);
    return D_FMA((float)e, 0x1.62e430p-1f, lm);   // e ln 2 + ln m
}

// Quadratic form q = d^T A d of a pixel offset d = (dx, dy) for the conic
// A = [[ca, cb], [cb, cc]]:  q = dx (ca dx + 2 cb dy) + cc dy^2, formed as
// a = ca dx + cb dy (fma), a = cb dy + a (fma), q = dx a + (cc dy) dy (fma).
__device__ __forceinline__ float dec_quad(float ca, float cb, float cc, float dx, float dy) {
    float a = D_FMA(ca, dx, D_MUL(cb, dy));
    a = D_FMA(cb, dy, a);
    return D_FMA(dx, a, D_MUL(D_MUL(cc, dy), dy));
}

// What the decisions need of one Gaussian in one view.
struct DecRec {
    float px, py;      // pixel-space centre
    float ca, cb, cc;  // conic (inverse of Sigma2D incl. the low-pass)
    float sxx, syy;    // Sigma2D diagonal incl. the low-pass
    float k2;          // det Sigma2D / syy^2 (row extent of the support ellipse)
    float l, lmax;     // thresholds of q (composited / clamped)
    float rx, ry;      // half extents of the support box, padded
};

// The projection of one visible Gaussian (camera depth tz >= near_z, sigma >=
// alpha_min), in this order:
//   t_x, t_y = V_r0,1 . p + t (fma chains, p_z term innermost); itz = 1 / tz;
//   tau = clamp(t / tz, +-L); J = [[fx itz, 0, -(fx tau_x) itz], [0, fy itz, -(fy tau_y) itz]];
//   T = J Wr (row a: J_a0 W_0j (+) J_a2 W_2j as fma(J_a0, W, J_a2 W));
//   q normalised by 1 / sqrt(q.q); R from the normalised quaternion;
//   m_a,j = (T R)_aj (fma chains); Sigma2D = sum_j s_j^2 m_.j m_.j^T;
//   det by Cauchy-Binet (a sum of non-negative terms) plus the low-pass terms;
//   conic = adj / det; centre = fma(fx t_x, itz, cx);
//   l = 2 ln(sigma / alpha_min), lmax = 2 ln(sigma / alpha_max) or -1;
//   half extents sqrt(l Sigma_ii) 1.0005 + 0.02 (so FP32 rounding can only add
//   tiles: the box of the exact support lies inside).
// V: row-major [R | t] (12 floats); Lx, Ly: the frustum clamp of tau.
__device__ __forceinline__ DecRec dec_project(const float *V, float fx, float fy, float cx, float cy, float Lx,
                                              float Ly, float px, float py, float pz, float tz, float qw, float qx,
                                              float qy, float qz, float s0, float s1, float s2, float sigma,
                                              float lowpass, float alpha_min, float alpha_max) {
    DecRec r;
    const float tx = D_FMA(V[0], px, D_FMA(V[1], py, D_FMA(V[2], pz, V[3])));
    const float ty = D_FMA(V[4], px, D_FMA(V[5], py, D_FMA(V[6], pz, V[7])));
    const float itz = D_DIV(1.f, tz);
    const float taux = fminf(fmaxf(D_MUL(tx, itz), -Lx), Lx);
    const float tauy = fminf(fmaxf(D_MUL(ty, itz), -Ly), Ly);
    const float j00 = D_MUL(fx, itz), j02 = D_MUL(D_MUL(-fx, taux), itz);
    const float j11 = D_MUL(fy, itz), j12 = D_MUL(D_MUL(-fy, tauy), itz);
    float T0[3], T1[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T0[j] = D_FMA(j00, V[j], D_MUL(j02, V[8 + j]));
        T1[j] = D_FMA(j11, V[4 + j], D_MUL(j12, V[8 + j]));
    }
    const float qq = D_FMA(qw, qw, D_FMA(qx, qx, D_FMA(qy, qy, D_MUL(qz, qz))));
    const float qn = D_DIV(1.f, D_SQRT(qq));
    const float w = D_MUL(qw, qn), x = D_MUL(qx, qn), y = D_MUL(qy, qn), z = D_MUL(qz, qn);
    float R[3][3];
    R[0][0] = D_SUB(1.f, D_MUL(2.f, D_FMA(y, y, D_MUL(z, z))));
    R[0][1] = D_MUL(2.f, D_SUB(D_MUL(x, y), D_MUL(w, z)));
    R[0][2] = D_MUL(2.f, D_ADD(D_MUL(x, z), D_MUL(w, y)));
    R[1][0] = D_MUL(2.f, D_ADD(D_MUL(x, y), D_MUL(w, z)));
    R[1][1] = D_SUB(1.f, D_MUL(2.f, D_FMA(x, x, D_MUL(z, z))));
    R[1][2] = D_MUL(2.f, D_SUB(D_MUL(y, z), D_MUL(w, x)));
    R[2][0] = D_MUL(2.f, D_SUB(D_MUL(x, z), D_MUL(w, y)));
    R[2][1] = D_MUL(2.f, D_ADD(D_MUL(y, z), D_MUL(w, x)));
    R[2][2] = D_SUB(1.f, D_MUL(2.f, D_FMA(x, x, D_MUL(y, y))));
    const float ss[3] = {D_MUL(s0, s0), D_MUL(s1, s1), D_MUL(s2, s2)};
    float m0[3], m1[3];
    float sxx = 0.f, sxy = 0.f, syy = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        m0[j] = D_FMA(T0[0], R[0][j], D_FMA(T0[1], R[1][j], D_MUL(T0[2], R[2][j])));
        m1[j] = D_FMA(T1[0], R[0][j], D_FMA(T1[1], R[1][j], D_MUL(T1[2], R[2][j])));
        const float a0 = D_MUL(ss[j], m0[j]);
        sxx = D_FMA(a0, m0[j], sxx);
        sxy = D_FMA(a0, m1[j], sxy);
        syy = D_FMA(D_MUL(ss[j], m1[j]), m1[j], syy);
    }
    // det(A + l I) = det A + l tr A + l^2, det A = sum_{i<j} s_i^2 s_j^2 (m_i x m_j)^2
    float detA = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i + 1; j < 3; ++j) {
            const float cr = D_FMA(m0[i], m1[j], -D_MUL(m1[i], m0[j]));
            detA = D_FMA(D_MUL(D_MUL(ss[i], ss[j]), cr), cr, detA);
        }
    const float det = D_ADD(D_ADD(detA, D_MUL(lowpass, D_ADD(sxx, syy))), D_MUL(lowpass, lowpass));
    sxx = D_ADD(sxx, lowpass);
    syy = D_ADD(syy, lowpass);
    const float idet = D_DIV(1.f, det);
    r.ca = D_MUL(syy, idet);
    r.cb = D_MUL(-sxy, idet);
    r.cc = D_MUL(sxx, idet);
    r.sxx = sxx;
    r.syy = syy;
    r.k2 = D_DIV(det, D_MUL(syy, syy));
    r.px = D_FMA(D_MUL(fx, tx), itz, cx);
    r.py = D_FMA(D_MUL(fy, ty), itz, cy);
    r.l = D_MUL(2.f, dec_ln(D_DIV(sigma, alpha_min)));
    r.lmax = sigma > alpha_max ? D_MUL(2.f, dec_ln(D_DIV(sigma, alpha_max))) : -1.f;
    r.rx = D_FMA(D_SQRT(fmaxf(D_MUL(r.l, sxx), 0.f)), 1.0005f, 0.02f);
    r.ry = D_FMA(D_SQRT(fmaxf(D_MUL(r.l, syy), 0.f)), 1.0005f, 0.02f);
    return r;
}

// ----------------------------------------------------- support ellipse per tile row
// The support { d : q(d) <= l } is, row by row (y relative to the centre),
// |x - k1 y| <= sqrt(k2 (ry^2 - y^2)) with k1 = Sigma_xy / Sigma_yy = -cb / ca,
// k2 = det Sigma / Sigma_yy^2 and ry^2 = l Sigma_yy (ry padded as the box).
// Over the pixel rows of one tile row the largest x is reached at the row
// nearest the ellipse's rightmost point (y* = k1 ry / sqrt(k2 + k1^2); x is
// concave in y) and the smallest at the row nearest -y*.  A margin of 1e-3 of
// the extents + 0.05 px keeps every tile that holds a pixel with q <= l, so
// the lists cover every composited term (tested against brute force).
struct SupportRows {
    float px, py, k1, k2, ry, ystar, marg;
};

__device__ __forceinline__ SupportRows support_rows(float px, float py, float ca, float cb, float k2, float ry) {
    SupportRows s;
    s.px = px;
    s.py = py;
    s.k2 = k2;
    s.ry = ry;
    s.k1 = D_DIV(-cb, ca);
    s.ystar = D_DIV(D_MUL(s.k1, ry), D_SQRT(D_FMA(s.k1, s.k1, k2)));
    s.marg = D_FMA(1e-3f, D_MUL(D_ADD(fabsf(s.k1), D_SQRT(k2)), ry), 0.05f);
    return s;
}

// The support over the pixel rows [y0, y0 + t) of a tile row: ok when some
// integer pixel row lies in its y-extent, and then the integer pixel columns
// [ceil(xl), floor(xr)] it may reach in that band (one computation serves
// every tile of the row).
struct SupportRow {
    bool ok;
    float cl, cr;
};

__device__ __forceinline__ SupportRow support_row(const SupportRows &s, float y0, float tile) {
    SupportRow o;
    const float ylo = fmaxf(y0, ceilf(D_SUB(s.py, s.ry)));
    const float yhi = fminf(D_SUB(D_ADD(y0, tile), 1.f), floorf(D_ADD(s.py, s.ry)));
    o.ok = ylo <= yhi;
    o.cl = 1.f;
    o.cr = 0.f;
    if (!o.ok) return o;
    const float ya = D_SUB(ylo, s.py), yb = D_SUB(yhi, s.py);
    const float yr = fminf(fmaxf(s.ystar, ya), yb), yl = fminf(fmaxf(-s.ystar, ya), yb);
    const float r2 = D_MUL(s.ry, s.ry);
    const float hr = D_SQRT(fmaxf(D_MUL(s.k2, D_SUB(r2, D_MUL(yr, yr))), 0.f));
    const float hl = D_SQRT(fmaxf(D_MUL(s.k2, D_SUB(r2, D_MUL(yl, yl))), 0.f));
    const float xr = D_ADD(D_ADD(D_FMA(s.k1, yr, s.px), hr), s.marg);   // rightmost reach in the band
    const float xl = D_SUB(D_SUB(D_FMA(s.k1, yl, s.px), hl), s.marg);   // leftmost
    o.cl = ceilf(xl);
    o.cr = floorf(xr);
    return o;
}

// some integer pixel column of the tile [x0, x0 + t) lies in the row's range
__device__ __forceinline__ bool support_row_reaches(const SupportRow &o, float x0, float tile) {
    const float c0 = fmaxf(o.cl, x0);
    const float c1 = fminf(o.cr, D_SUB(D_ADD(x0, tile), 1.f));
    return o.ok && c0 <= c1;
}

// Does the support reach a pixel of the tile with pixel rows [y0, y0 + t) and
// columns [x0, x0 + t)?
__device__ __forceinline__ bool support_reaches(const SupportRows &s, float x0, float y0, float tile) {
    return support_row_reaches(support_row(s, y0, tile), x0, tile);
}
