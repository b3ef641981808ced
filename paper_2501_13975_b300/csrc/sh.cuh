// Real spherical-harmonic colour basis of degree <= 3 (App. A.2): values,
// gradients and Hessians of B_i Phi_i(r) as polynomials in the direction r.
// B_i are the orthonormal real-SH normalisations sqrt((2l+1)/(4 pi) ...),
// written out as literals, with the sign convention of the standard 3DGS
// colour model; Phi_i is the paper's polynomial list in its order.
#pragma once

__device__ __forceinline__ float sh_norm(int i) {
    switch (i) {
    case 0: return 0.28209479177387814f;
    case 1: case 2: case 3: return 0.4886025119029199f;
    case 4: return 1.0925484305920792f;
    case 5: return -1.0925484305920792f;
    case 6: return 0.31539156525252005f;
    case 7: return -1.0925484305920792f;
    case 8: return 0.5462742152960396f;
    case 9: return -0.5900435899266435f;
    case 10: return 2.890611442640554f;
    case 11: return -0.4570457994644658f;
    case 12: return 0.3731763325901154f;
    case 13: return -0.4570457994644658f;
    case 14: return 1.445305721320277f;
    default: return -0.5900435899266435f;
    }
}

// phi[i] = Phi_i(x, y, z) for i < S
__device__ __forceinline__ void sh_phi(int S, float x, float y, float z, float *phi) {
    phi[0] = 1.f;
    if (S <= 1) return;
    phi[1] = -y; phi[2] = z; phi[3] = -x;
    if (S <= 4) return;
    float xx = x * x, yy = y * y, zz = z * z;
    phi[4] = x * y; phi[5] = y * z; phi[6] = 2.f * zz - xx - yy; phi[7] = x * z; phi[8] = xx - yy;
    if (S <= 9) return;
    phi[9] = y * (3.f * xx - yy);
    phi[10] = x * y * z;
    phi[11] = y * (4.f * zz - xx - yy);
    phi[12] = z * (2.f * zz - 3.f * xx - 3.f * yy);
    phi[13] = x * (4.f * zz - xx - yy);
    phi[14] = z * (xx - yy);
    phi[15] = x * (xx - 3.f * yy);
}

// Accumulates sum_i w_i Phi_i into value f, gradient g[3] and Hessian
// hs[6] (xx xy xz yy yz zz) for coefficient weights w[i], i < S.
__device__ __forceinline__ void sh_poly_derivs(int S, const float *w, float x, float y, float z, float &f, float g[3],
                                               float hs[6]) {
    f = w[0];
    g[0] = g[1] = g[2] = 0.f;
    for (int i = 0; i < 6; ++i) hs[i] = 0.f;
    if (S <= 1) return;
    // degree 1: -y, z, -x
    f += -w[1] * y + w[2] * z - w[3] * x;
    g[0] += -w[3]; g[1] += -w[1]; g[2] += w[2];
    if (S <= 4) return;
    float xx = x * x, yy = y * y, zz = z * z;
    // xy
    f += w[4] * x * y; g[0] += w[4] * y; g[1] += w[4] * x; hs[1] += w[4];
    // yz
    f += w[5] * y * z; g[1] += w[5] * z; g[2] += w[5] * y; hs[4] += w[5];
    // 2z^2 - x^2 - y^2
    f += w[6] * (2.f * zz - xx - yy); g[0] += -2.f * w[6] * x; g[1] += -2.f * w[6] * y; g[2] += 4.f * w[6] * z;
    hs[0] += -2.f * w[6]; hs[3] += -2.f * w[6]; hs[5] += 4.f * w[6];
    // xz
    f += w[7] * x * z; g[0] += w[7] * z; g[2] += w[7] * x; hs[2] += w[7];
    // x^2 - y^2
    f += w[8] * (xx - yy); g[0] += 2.f * w[8] * x; g[1] += -2.f * w[8] * y; hs[0] += 2.f * w[8]; hs[3] += -2.f * w[8];
    if (S <= 9) return;
    // 3 x^2 y - y^3
    f += w[9] * y * (3.f * xx - yy);
    g[0] += 6.f * w[9] * x * y; g[1] += w[9] * (3.f * xx - 3.f * yy);
    hs[0] += 6.f * w[9] * y; hs[1] += 6.f * w[9] * x; hs[3] += -6.f * w[9] * y;
    // xyz
    f += w[10] * x * y * z;
    g[0] += w[10] * y * z; g[1] += w[10] * x * z; g[2] += w[10] * x * y;
    hs[1] += w[10] * z; hs[2] += w[10] * y; hs[4] += w[10] * x;
    // 4 y z^2 - x^2 y - y^3
    f += w[11] * y * (4.f * zz - xx - yy);
    g[0] += -2.f * w[11] * x * y; g[1] += w[11] * (4.f * zz - xx - 3.f * yy); g[2] += 8.f * w[11] * y * z;
    hs[0] += -2.f * w[11] * y; hs[1] += -2.f * w[11] * x; hs[3] += -6.f * w[11] * y; hs[4] += 8.f * w[11] * z;
    hs[5] += 8.f * w[11] * y;
    // 2 z^3 - 3 x^2 z - 3 y^2 z
    f += w[12] * z * (2.f * zz - 3.f * xx - 3.f * yy);
    g[0] += -6.f * w[12] * x * z; g[1] += -6.f * w[12] * y * z; g[2] += w[12] * (6.f * zz - 3.f * xx - 3.f * yy);
    hs[0] += -6.f * w[12] * z; hs[2] += -6.f * w[12] * x; hs[3] += -6.f * w[12] * z; hs[4] += -6.f * w[12] * y;
    hs[5] += 12.f * w[12] * z;
    // 4 x z^2 - x^3 - x y^2
    f += w[13] * x * (4.f * zz - xx - yy);
    g[0] += w[13] * (4.f * zz - 3.f * xx - yy); g[1] += -2.f * w[13] * x * y; g[2] += 8.f * w[13] * x * z;
    hs[0] += -6.f * w[13] * x; hs[1] += -2.f * w[13] * y; hs[2] += 8.f * w[13] * z; hs[3] += -2.f * w[13] * x;
    hs[5] += 8.f * w[13] * x;
    // x^2 z - y^2 z
    f += w[14] * z * (xx - yy);
    g[0] += 2.f * w[14] * x * z; g[1] += -2.f * w[14] * y * z; g[2] += w[14] * (xx - yy);
    hs[0] += 2.f * w[14] * z; hs[2] += 2.f * w[14] * x; hs[3] += -2.f * w[14] * z; hs[4] += -2.f * w[14] * y;
    // x^3 - 3 x y^2
    f += w[15] * x * (xx - 3.f * yy);
    g[0] += w[15] * (3.f * xx - 3.f * yy); g[1] += -6.f * w[15] * x * y;
    hs[0] += 6.f * w[15] * x; hs[1] += -6.f * w[15] * y; hs[3] += -6.f * w[15] * x;
}
