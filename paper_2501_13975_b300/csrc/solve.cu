// gs2_solve_step / gs2_apply_step: per-Gaussian damped local Newton steps
// (Eq. local_newton) and the group updates (Sec. 4.2).
//
// Damping (the paper fixes step size 1 and is silent on indefinite blocks):
// H + mu m I with m = mean |diag H|, mu = mu0 10^i, i = 0..tries, until the
// Cholesky factorisation has positive pivots; otherwise the step is 0 and the
// failure is counted.  A block with all-zero gradient and Hessian (no
// contributing pixel) gets a zero step.
//   position: 2x2 solve in U = [u_x, u_y] perpendicular to the primary view ray
//   rotation: scalar angle about the primary view ray
//   scaling:  2x2 solve in the row space of d lambda / d s (eigenvalues of the
//             primary view's projected covariance), update kept in [s/k, k s]
//   opacity:  scalar with the log barrier, fraction-to-boundary inside (0, 1)
//   colour:   S x S per channel from the factored per-view slots
// Trust radii (position 3 max(s), rotation pi/4, colour 2 sqrt(pi) per
// channel) scale down over-long steps; non-finite steps become 0 (failed).
// One thread per Gaussian (per Gaussian and channel for colour); blocks of
// size <= 3 live in registers, the 16x16 colour factor in local memory.
#include "common.cuh"

template <int NMAX, typename T, typename TI = float>
__device__ int damped_solve_t(int N, const TI *H, const TI *g, float mu0, int tries, T *x, float *kappa) {
    T m = 0, gz = 0;
    for (int i = 0; i < N; ++i) {
        m += fabs((T)H[i * N + i]);
        gz += fabs((T)g[i]);
        x[i] = 0;
    }
    for (int i = 0; i < N * N; ++i) gz += fabs((T)H[i]);
    if (kappa) *kappa = 1.f;
    if (gz == 0) return 2;
    m /= (T)N;
    T mu = (T)mu0;
    T L[NMAX * NMAX];
    for (int att = 0; att <= tries; ++att, mu *= 10) {
        bool ok = true;
        for (int j = 0; j < N && ok; ++j) {
            T d = (T)H[j * N + j] + mu * m;
            for (int k = 0; k < j; ++k) d -= L[j * N + k] * L[j * N + k];
            if (!(d > 0)) {
                ok = false;
                break;
            }
            const T ljj = sqrt(d);
            L[j * N + j] = ljj;
            const T il = 1 / ljj;
            for (int i = j + 1; i < N; ++i) {
                T sm = (T)H[i * N + j];
                for (int k = 0; k < j; ++k) sm -= L[i * N + k] * L[j * N + k];
                L[i * N + j] = sm * il;
            }
        }
        if (!ok) continue;
        T y[NMAX];
        for (int i = 0; i < N; ++i) {
            T sm = -(T)g[i];
            for (int k = 0; k < i; ++k) sm -= L[i * N + k] * y[k];
            y[i] = sm / L[i * N + i];
        }
        for (int i = N - 1; i >= 0; --i) {
            T sm = y[i];
            for (int k = i + 1; k < N; ++k) sm -= L[k * N + i] * x[k];
            x[i] = sm / L[i * N + i];
        }
        if (kappa) {   // condition estimate from the factor: (max L_ii / min L_ii)^2
            T lo = L[0], hi = L[0];
            for (int i = 1; i < N; ++i) {
                lo = fmin(lo, L[i * N + i]);
                hi = fmax(hi, L[i * N + i]);
            }
            *kappa = (float)((hi / lo) * (hi / lo));
        }
        return 0;
    }
    for (int i = 0; i < N; ++i) x[i] = 0;
    return 1;
}

// FP32 damped solve; with mixed precision (precision = 1) a block whose
// condition estimate exceeds 1e6 is solved again in FP64.
// resolves (may be NULL) counts the blocks solved again in FP64.
template <int NMAX>
__device__ int damped_solve(int N, const float *H, const float *g, float mu0, int tries, float *x, int precision,
                            unsigned long long *resolves) {
    float kappa = 1.f;
    int st = damped_solve_t<NMAX, float>(N, H, g, mu0, tries, x, &kappa);
    if (precision != 0 && st != 2 && (st == 1 || kappa > 1e6f)) {
        double xd[NMAX];
        st = damped_solve_t<NMAX, double>(N, H, g, mu0, tries, xd, nullptr);
        for (int i = 0; i < N; ++i) x[i] = (float)xd[i];
        if (resolves) atomicAdd(resolves, 1ull);
    }
    return st;
}

// Trust radius: a step longer than `radius` is scaled down to it (direction
// kept); a non-finite step becomes zero and reports failure.
template <typename T>
__device__ __forceinline__ bool trust_scale_t(int N, T *x, T radius) {
    T nn = 0;
    for (int i = 0; i < N; ++i) nn += x[i] * x[i];
    nn = sqrt(nn);
    if (!isfinite(nn)) {
        for (int i = 0; i < N; ++i) x[i] = 0;
        return true;
    }
    if (nn > radius) {
        const T f = radius / nn;
        for (int i = 0; i < N; ++i) x[i] *= f;
    }
    return false;
}
__device__ __forceinline__ bool trust_scale(int N, float *x, float radius) { return trust_scale_t<float>(N, x, radius); }

__device__ __forceinline__ void unit_dir(const DevCam &cam, const float p[3], float r[3]) {
    r[0] = p[0] - cam.o[0];
    r[1] = p[1] - cam.o[1];
    r[2] = p[2] - cam.o[2];
    const float in = rsqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    r[0] *= in; r[1] *= in; r[2] *= in;
}

// Basis U = [u_x, u_y] of the plane perpendicular to the primary view ray r
// and the reduced problem g_v = U^T g, H_v = U^T H U, in the precision T.
template <typename T>
__device__ __forceinline__ void pos_reduce(const DevCam &pr, const float p[3], const float g[3], const float (&Hm)[3][3],
                                           T ux[3], T uy[3], T gv[2], T Hv[4]) {
    T r[3] = {(T)p[0] - (T)pr.o[0], (T)p[1] - (T)pr.o[1], (T)p[2] - (T)pr.o[2]};
    const T in = (T)1 / sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    r[0] *= in; r[1] *= in; r[2] *= in;
    T e[3] = {0, 1, 0};
    if (fabs(r[1]) > (T)0.999) { e[0] = 1; e[1] = 0; }
    const T d = r[0] * e[0] + r[1] * e[1] + r[2] * e[2];
    T v[3] = {e[0] - d * r[0], e[1] - d * r[1], e[2] - d * r[2]};
    const T un = (T)1 / sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int i = 0; i < 3; ++i) uy[i] = v[i] * un;
    ux[0] = r[1] * uy[2] - r[2] * uy[1];
    ux[1] = r[2] * uy[0] - r[0] * uy[2];
    ux[2] = r[0] * uy[1] - r[1] * uy[0];
    const T *U[2] = {ux, uy};
    for (int a = 0; a < 2; ++a) {
        gv[a] = U[a][0] * (T)g[0] + U[a][1] * (T)g[1] + U[a][2] * (T)g[2];
        for (int b = 0; b < 2; ++b) {
            T acc = 0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) acc += U[a][i] * (T)Hm[i][j] * U[b][j];
            Hv[a * 2 + b] = acc;
        }
    }
}

// Position step: the damped 2x2 solve in the plane perpendicular to the view
// ray.  With mixed precision a block whose FP32 condition estimate exceeds
// 1e6 (or whose FP32 ladder failed) is solved again with its basis,
// reduction, factorisation and step all in FP64.
__global__ void k_solve_pos(DevScene sc, DevCam pr, const float *__restrict__ B, float mu0, int tries, float trust,
                            float *step, int32_t *nfail, int prec, unsigned long long *resolves,
                            const float *__restrict__ rho) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = sc.n;
    if (k >= n) return;
    if (rho) mu0 *= rho[k];   // learned per-Gaussian damping multiplier
    const float p[3] = {sc.mean[k], sc.mean[n + k], sc.mean[2 * n + k]};
    const float g[3] = {B[k], B[n + k], B[2 * n + k]};
    const float h00 = B[3 * n + k], h01 = B[4 * n + k], h02 = B[5 * n + k], h11 = B[6 * n + k], h12 = B[7 * n + k],
                h22 = B[8 * n + k];
    const float Hm[3][3] = {{h00, h01, h02}, {h01, h11, h12}, {h02, h12, h22}};
    float ux[3], uy[3], gv[2], Hv[4], dv[2], kappa = 1.f;
    pos_reduce<float>(pr, p, g, Hm, ux, uy, gv, Hv);
    int st = damped_solve_t<2, float>(2, Hv, gv, mu0, tries, dv, &kappa);
    const float smax = fmaxf(sc.scale[k], fmaxf(sc.scale[n + k], sc.scale[2 * n + k]));
    float dp[3];
    if (prec != 0 && st != 2 && (st == 1 || kappa > 1e6f)) {
        double uxd[3], uyd[3], gvd[2], Hvd[4], dvd[2];
        pos_reduce<double>(pr, p, g, Hm, uxd, uyd, gvd, Hvd);
        st = damped_solve_t<2, double, double>(2, Hvd, gvd, mu0, tries, dvd, nullptr);
        if (resolves) atomicAdd(resolves, 1ull);
        if (st == 0 && trust_scale_t<double>(2, dvd, (double)trust * (double)smax)) st = 1;
        for (int i = 0; i < 3; ++i) dp[i] = (float)(uxd[i] * dvd[0] + uyd[i] * dvd[1]);
    } else {
        if (st == 0 && trust_scale(2, dv, trust * smax)) st = 1;
        for (int i = 0; i < 3; ++i) dp[i] = ux[i] * dv[0] + uy[i] * dv[1];
    }
    if (st == 1 && nfail) atomicAdd(nfail, 1);
    for (int i = 0; i < 3; ++i) step[(size_t)i * n + k] = dp[i];
}

__global__ void k_solve_scalar(int n, const float *__restrict__ B, float mu0, int tries, float trust, float *step,
                               int32_t *nfail, int prec, unsigned long long *resolves) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float g = B[k], h = B[n + k];
    float x;
    int st = damped_solve<1>(1, &h, &g, mu0, tries, &x, prec, resolves);
    if (st == 0 && trust_scale(1, &x, trust)) st = 1;
    if (st == 1 && nfail) atomicAdd(nfail, 1);
    step[k] = x;
}

__global__ void k_solve_opacity(DevScene sc, const float *__restrict__ B, float mu0, int tries, float barrier,
                                float tau, float *step, int32_t *nfail, int prec, unsigned long long *resolves) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = sc.n;
    if (k >= n) return;
    const float sg = sc.opacity[k];
    float g = B[k], h = B[n + k], x = 0.f;
    int st = 2;
    if (!(g == 0.f && h == 0.f)) {
        g += barrier * (-1.f / sg + 1.f / (1.f - sg));
        h += barrier * (1.f / (sg * sg) + 1.f / ((1.f - sg) * (1.f - sg)));
        st = damped_solve<1>(1, &h, &g, mu0, tries, &x, prec, resolves);
        if (st == 0 && trust_scale(1, &x, INFINITY)) st = 1;
    }
    if (st == 1 && nfail) atomicAdd(nfail, 1);
    // fraction-to-boundary on the increment itself: x in [-tau sigma, tau (1 - sigma)]
    const float xc = fminf(fmaxf(x, -tau * sg), tau * (1.f - sg));
    step[k] = (st == 0) ? xc : 0.f;
}

// Scaling reduction in the precision T: lambda_i = sum_j (V M)_ij^2 s_j^2 with
// M = J Wr R of the primary view and V the eigenvectors of M diag(s^2) M^T;
// Tt = d lambda / d s, Q = Tt^T (Tt Tt^T)^-1 (3x2), g_l = Q^T g, H_l = Q^T H Q.
// Returns false where the reduction is undefined (behind the primary camera,
// or rows of Tt (near-)parallel: relative det(Tt Tt^T) < 1e-6).
template <typename T>
__device__ __forceinline__ bool scale_reduce(const DevCam &pr, const float p[3], const float s[3], const float q4[4],
                                             const float g[3], const float (&Hm)[3][3], T (&Q)[3][2], T gl[2],
                                             T Hl[4]) {
    const float *V = pr.V;
    T t[3];
    for (int i = 0; i < 3; ++i)
        t[i] = (T)V[i * 4] * (T)p[0] + (T)V[i * 4 + 1] * (T)p[1] + (T)V[i * 4 + 2] * (T)p[2] + (T)V[i * 4 + 3];
    const T iz = (T)1 / t[2];
    const T Lx = (T)pr.Lx, Ly = (T)pr.Ly;
    const T taux = fmin(fmax(t[0] * iz, -Lx), Lx), tauy = fmin(fmax(t[1] * iz, -Ly), Ly);
    const T fx = (T)pr.fx, fy = (T)pr.fy;
    const T J[2][3] = {{fx * iz, (T)0, -fx * taux * iz}, {(T)0, fy * iz, -fy * tauy * iz}};
    T qw = (T)q4[0], qx = (T)q4[1], qy = (T)q4[2], qz = (T)q4[3];
    const T qn = (T)1 / sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
    qw *= qn; qx *= qn; qy *= qn; qz *= qn;
    const T R[3][3] = {{1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)},
                       {2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)},
                       {2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)}};
    T M[2][3];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b) {
            T acc = 0;
            for (int i = 0; i < 3; ++i) {
                const T wr = (T)V[i * 4] * R[0][b] + (T)V[i * 4 + 1] * R[1][b] + (T)V[i * 4 + 2] * R[2][b];
                acc += J[a][i] * wr;
            }
            M[a][b] = acc;
        }
    T A00 = 0, A01 = 0, A11 = 0;
    for (int j = 0; j < 3; ++j) {
        const T s2 = (T)s[j] * (T)s[j];
        A00 += M[0][j] * M[0][j] * s2;
        A01 += M[0][j] * M[1][j] * s2;
        A11 += M[1][j] * M[1][j] * s2;
    }
    const T phi = (T)0.5 * atan2(2 * A01, A00 - A11);
    const T c = cos(phi), sn = sin(phi);
    T Tt[2][3];
    for (int j = 0; j < 3; ++j) {
        const T a = c * M[0][j] + sn * M[1][j];
        const T b = -sn * M[0][j] + c * M[1][j];
        Tt[0][j] = 2 * a * a * (T)s[j];
        Tt[1][j] = 2 * b * b * (T)s[j];
    }
    T G00 = 0, G01 = 0, G11 = 0;
    for (int j = 0; j < 3; ++j) {
        G00 += Tt[0][j] * Tt[0][j];
        G01 += Tt[0][j] * Tt[1][j];
        G11 += Tt[1][j] * Tt[1][j];
    }
    const T det = G00 * G11 - G01 * G01;
    if (!(det > (T)1e-30) || !(det > (T)1e-6 * G00 * G11)) return false;
    const T I00 = G11 / det, I01 = -G01 / det, I11 = G00 / det;
    for (int j = 0; j < 3; ++j) {
        Q[j][0] = Tt[0][j] * I00 + Tt[1][j] * I01;
        Q[j][1] = Tt[0][j] * I01 + Tt[1][j] * I11;
    }
    for (int a = 0; a < 2; ++a) {
        gl[a] = Q[0][a] * (T)g[0] + Q[1][a] * (T)g[1] + Q[2][a] * (T)g[2];
        for (int b = 0; b < 2; ++b) {
            T acc = 0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) acc += Q[i][a] * (T)Hm[i][j] * Q[j][b];
            Hl[a * 2 + b] = acc;
        }
    }
    return true;
}

// Scaling step: damped 2x2 solve in the row space of Tt, update kept in
// [s / trust, trust s].  With mixed precision a block whose FP32 condition
// estimate exceeds 1e6 (or whose FP32 ladder failed) is solved again with its
// reduction, factorisation and step in FP64.
__global__ void k_solve_scale(DevScene sc, DevCam pr, const float *__restrict__ B, float mu0, int tries,
                              float near_z, float trust, float *step, int32_t *nfail, int prec,
                              unsigned long long *resolves, const float *__restrict__ rho) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = sc.n;
    if (k >= n) return;
    if (rho) mu0 *= rho[k];   // learned per-Gaussian damping multiplier
    const float g[3] = {B[k], B[n + k], B[2 * n + k]};
    float Hs[6];
    bool zero = g[0] == 0.f && g[1] == 0.f && g[2] == 0.f;
    for (int i = 0; i < 6; ++i) {
        Hs[i] = B[(size_t)(3 + i) * n + k];
        zero = zero && Hs[i] == 0.f;
    }
    for (int i = 0; i < 3; ++i) step[(size_t)i * n + k] = 0.f;
    if (zero) return;
    const float p[3] = {sc.mean[k], sc.mean[n + k], sc.mean[2 * n + k]};
    const float s[3] = {sc.scale[k], sc.scale[n + k], sc.scale[2 * n + k]};
    const float q4[4] = {sc.quat[k], sc.quat[n + k], sc.quat[2 * n + k], sc.quat[3 * n + k]};
    const float *V = pr.V;
    double dz = (double)V[8] * (double)p[0];
    dz = dz + (double)V[9] * (double)p[1];
    dz = dz + (double)V[10] * (double)p[2];
    dz = dz + (double)V[11];
    if (!(dz >= (double)near_z)) return;
    const float Hm[3][3] = {{Hs[0], Hs[1], Hs[2]}, {Hs[1], Hs[3], Hs[4]}, {Hs[2], Hs[4], Hs[5]}};
    float Q[3][2], gl[2], Hl[4], dl[2], kappa = 1.f;
    if (!scale_reduce<float>(pr, p, s, q4, g, Hm, Q, gl, Hl)) return;
    int st = damped_solve_t<2, float>(2, Hl, gl, mu0, tries, dl, &kappa);
    float ds[3];
    if (prec != 0 && st != 2 && (st == 1 || kappa > 1e6f)) {
        double Qd[3][2], gld[2], Hld[4], dld[2];
        if (resolves) atomicAdd(resolves, 1ull);
        if (!scale_reduce<double>(pr, p, s, q4, g, Hm, Qd, gld, Hld)) return;
        st = damped_solve_t<2, double, double>(2, Hld, gld, mu0, tries, dld, nullptr);
        if (st == 0 && trust_scale_t<double>(2, dld, (double)INFINITY)) st = 1;
        for (int i = 0; i < 3; ++i) ds[i] = (float)(Qd[i][0] * dld[0] + Qd[i][1] * dld[1]);
    } else {
        if (st == 0 && trust_scale(2, dl, INFINITY)) st = 1;
        for (int i = 0; i < 3; ++i) ds[i] = Q[i][0] * dl[0] + Q[i][1] * dl[1];
    }
    if (st == 1 && nfail) atomicAdd(nfail, 1);
    // s + ds stays in [s / trust, s trust], clamped on the increment
    for (int i = 0; i < 3; ++i) step[(size_t)i * n + k] = fminf(fmaxf(ds[i], s[i] / trust - s[i]), s[i] * trust - s[i]);
}

__global__ void k_solve_color(DevScene sc, const float *__restrict__ B, int n_views, float mu0, int tries,
                              float trust, float *step, int32_t *nfail, int prec, unsigned long long *resolves,
                              const float *__restrict__ rho) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = sc.n, S = sc.S;
    if (idx >= 3 * n) return;
    const int ch = idx / n, k = idx % n;
    if (rho) mu0 *= rho[k];   // learned per-Gaussian damping multiplier
    float H[GS2_MAX_SH * GS2_MAX_SH], g[GS2_MAX_SH], x[GS2_MAX_SH];
    for (int i = 0; i < S * S; ++i) H[i] = 0.f;
    for (int i = 0; i < S; ++i) g[i] = 0.f;
    const size_t slot = (size_t)(6 + S) * n;
    for (int v = 0; v < n_views; ++v) {
        const float *Bv = B + v * slot;
        const float a = Bv[(size_t)ch * n + k], s = Bv[(size_t)(3 + ch) * n + k];
        if (a == 0.f && s == 0.f) continue;
        float b[GS2_MAX_SH];
        for (int i = 0; i < S; ++i) b[i] = Bv[(size_t)(6 + i) * n + k];
        for (int i = 0; i < S; ++i) {
            g[i] += a * b[i];
            for (int j = 0; j < S; ++j) H[i * S + j] += s * b[i] * b[j];
        }
    }
    int st = damped_solve<GS2_MAX_SH>(S, H, g, mu0, tries, x, prec, resolves);
    if (st == 0 && trust_scale(S, x, trust)) st = 1;
    if (st == 1 && nfail) atomicAdd(nfail, 1);
    for (int i = 0; i < S; ++i) step[(size_t)(ch * S + i) * n + k] = x[i];
}

// Colour solve in the range of the view basis (exact algebra, no dense block):
// H_ch = sum_v s_v b_v b_v^T = B S B^T with B = [b_1 .. b_V] (S x V, V <= 4).
// With B = Q R (modified Gram-Schmidt, re-orthogonalised; Q has r <= V
// orthonormal columns), H + d I = Q (d I_r + R S R^T) Q^T + d (I - Q Q^T), so
// the damped block is positive definite iff d I_r + K (K = R S R^T) is, and
// d > 0 when r < S; g = B a = Q R a lies in range(Q), hence
// x = -Q (d I_r + K)^{-1} R a.  m = mean |diag H| as for the dense block.
// Q and R are shared by the three channels.  One thread per Gaussian.
#define QR_VMAX 4

template <int S, typename T>
__device__ void qr_color_solve(const float (&a)[QR_VMAX][3], const float (&s)[QR_VMAX][3], const float (&b)[QR_VMAX][S],
                               int n_views, float mu0, int tries, float trust, unsigned chan_mask, float (&out)[3][S],
                               int (&status)[3], float (&kappa)[3]) {
    constexpr int VMAX = QR_VMAX;
    T q[VMAX][S];
#pragma unroll
    for (int v = 0; v < VMAX; ++v)
#pragma unroll
        for (int i = 0; i < S; ++i) q[v][i] = (T)b[v][i];
    // m per channel from diag H = sum_v s_v b_v^2
    T m[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T acc = 0;
#pragma unroll
        for (int i = 0; i < S; ++i) {
            T d = 0;
#pragma unroll
            for (int v = 0; v < VMAX; ++v) d += (T)s[v][c] * q[v][i] * q[v][i];
            acc += fabs(d);
        }
        m[c] = acc / (T)S;
    }
    // modified Gram-Schmidt with one re-orthogonalisation: B = Q R
    T R[VMAX][VMAX];
    bool keep[VMAX];
#pragma unroll
    for (int v = 0; v < VMAX; ++v) {
        keep[v] = false;
#pragma unroll
        for (int u = 0; u < VMAX; ++u) R[u][v] = 0;
        T b2 = 0;
#pragma unroll
        for (int i = 0; i < S; ++i) b2 += q[v][i] * q[v][i];
#pragma unroll
        for (int pass = 0; pass < 2; ++pass)
#pragma unroll
            for (int u = 0; u < VMAX; ++u) {
                if (u >= v || !keep[u]) continue;
                T d = 0;
#pragma unroll
                for (int i = 0; i < S; ++i) d += q[u][i] * q[v][i];
                R[u][v] += d;
#pragma unroll
                for (int i = 0; i < S; ++i) q[v][i] -= d * q[u][i];
            }
        T nn = 0;
#pragma unroll
        for (int i = 0; i < S; ++i) nn += q[v][i] * q[v][i];
        nn = sqrt(nn);
        keep[v] = (v < n_views) && nn > (T)1e-5 * sqrt(b2) && nn > 0;
        R[v][v] = keep[v] ? nn : (T)0;
        const T inv = keep[v] ? (T)1 / nn : (T)0;
#pragma unroll
        for (int i = 0; i < S; ++i) q[v][i] *= inv;
    }
    int r = 0;
#pragma unroll
    for (int v = 0; v < VMAX; ++v) r += keep[v] ? 1 : 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (!(chan_mask & (1u << c))) continue;
        T x[S];
#pragma unroll
        for (int i = 0; i < S; ++i) x[i] = 0;
        kappa[c] = 1.f;
        bool zero = true;
#pragma unroll
        for (int v = 0; v < VMAX; ++v) zero = zero && a[v][c] == 0.f && s[v][c] == 0.f;
        int st = 2;
        if (!zero) {
            T K[VMAX][VMAX], ra[VMAX];   // K = R S R^T, R a
#pragma unroll
            for (int u = 0; u < VMAX; ++u) {
                T acc = 0;
#pragma unroll
                for (int v = 0; v < VMAX; ++v) acc += R[u][v] * (T)a[v][c];
                ra[u] = acc;
#pragma unroll
                for (int w = 0; w < VMAX; ++w) {
                    T kk = 0;
#pragma unroll
                    for (int v = 0; v < VMAX; ++v) kk += R[u][v] * (T)s[v][c] * R[w][v];
                    K[u][w] = kk;
                }
            }
            st = 1;
            T mu = (T)mu0;
            for (int att = 0; att <= tries && st == 1; ++att, mu *= 10) {
                const T dl = mu * m[c];
                if (r < S && !(dl > 0)) continue;
                T L[VMAX][VMAX];
                bool ok = true;
#pragma unroll
                for (int j = 0; j < VMAX; ++j) {
                    if (!keep[j] || !ok) continue;
                    T d = dl + K[j][j];
#pragma unroll
                    for (int t = 0; t < VMAX; ++t)
                        if (t < j && keep[t]) d -= L[j][t] * L[j][t];
                    if (!(d > 0)) {
                        ok = false;
                        continue;
                    }
                    L[j][j] = sqrt(d);
#pragma unroll
                    for (int i = 0; i < VMAX; ++i) {
                        if (i <= j || !keep[i]) continue;
                        T sm = K[i][j];
#pragma unroll
                        for (int t = 0; t < VMAX; ++t)
                            if (t < j && keep[t]) sm -= L[i][t] * L[j][t];
                        L[i][j] = sm / L[j][j];
                    }
                }
                if (!ok) continue;
                T y[VMAX], z[VMAX], lo = (T)1e30, hi = 0;
#pragma unroll
                for (int i = 0; i < VMAX; ++i) {
                    if (!keep[i]) { y[i] = 0; continue; }
                    lo = fmin(lo, L[i][i]);
                    hi = fmax(hi, L[i][i]);
                    T sm = -ra[i];
#pragma unroll
                    for (int t = 0; t < VMAX; ++t)
                        if (t < i && keep[t]) sm -= L[i][t] * y[t];
                    y[i] = sm / L[i][i];
                }
#pragma unroll
                for (int i = VMAX - 1; i >= 0; --i) {
                    if (!keep[i]) { z[i] = 0; continue; }
                    T sm = y[i];
#pragma unroll
                    for (int t = 0; t < VMAX; ++t)
                        if (t > i && keep[t]) sm -= L[t][i] * z[t];
                    z[i] = sm / L[i][i];
                }
                if (r < S) lo = fmin(lo, sqrt(dl));   // the complement contributes d
                kappa[c] = (hi > 0 && lo > 0) ? (float)((hi / lo) * (hi / lo)) : 1e30f;
#pragma unroll
                for (int i = 0; i < S; ++i) {
                    T acc = 0;
#pragma unroll
                    for (int u = 0; u < VMAX; ++u) acc += q[u][i] * z[u];
                    x[i] = acc;
                }
                st = 0;
            }
        }
#pragma unroll
        for (int i = 0; i < S; ++i) out[c][i] = (float)x[i];
        if (st == 0 && trust_scale(S, out[c], trust)) st = 1;
        if (st != 0)
#pragma unroll
            for (int i = 0; i < S; ++i) out[c][i] = 0.f;
        status[c] = st;
    }
}

// Colour solve in the range of the view basis (exact algebra, no dense block):
// H_ch = sum_v s_v b_v b_v^T = B S B^T with B = [b_1 .. b_V] (S x V, V <= 4).
// With B = Q R (modified Gram-Schmidt, re-orthogonalised; Q has r <= V
// orthonormal columns), H + d I = Q (d I_r + R S R^T) Q^T + d (I - Q Q^T), so
// the damped block is positive definite iff d I_r + K (K = R S R^T) is, and
// d > 0 when r < S; g = B a = Q R a lies in range(Q), hence
// x = -Q (d I_r + K)^{-1} R a.  m = mean |diag H| as for the dense block.
// Q and R are shared by the three channels.  One thread per Gaussian.  With
// mixed precision, a channel whose condition estimate exceeds 1e6 (or whose
// damping ladder failed) is solved again in FP64.
template <int S>
__device__ __forceinline__ void load_color_slots(const float *__restrict__ B, int n, int k, int n_views,
                                                 float (&a)[QR_VMAX][3], float (&s)[QR_VMAX][3],
                                                 float (&b)[QR_VMAX][S]) {
    const size_t slot = (size_t)(6 + S) * n;
#pragma unroll
    for (int v = 0; v < QR_VMAX; ++v) {
        const bool on = v < n_views;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a[v][c] = on ? B[v * slot + (size_t)c * n + k] : 0.f;
            s[v][c] = on ? B[v * slot + (size_t)(3 + c) * n + k] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < S; ++i) b[v][i] = on ? B[v * slot + (size_t)(6 + i) * n + k] : 0.f;
    }
}

// FP32 pass: one thread per Gaussian.  With mixed precision it leaves in
// flags[k] the channels whose condition estimate exceeds 1e6 or whose ladder
// failed; k_solve_color_qr64 solves those again in FP64.
template <int S>
__global__ void __launch_bounds__(128) k_solve_color_qr(DevScene sc, const float *__restrict__ B, int n_views,
                                                        float mu0, int tries, float trust, float *step,
                                                        int32_t *nfail, int prec, uint8_t *flags,
                                                        const float *__restrict__ rho) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = sc.n;
    if (k >= n) return;
    if (rho) mu0 *= rho[k];   // learned per-Gaussian damping multiplier
    float a[QR_VMAX][3], s[QR_VMAX][3], b[QR_VMAX][S];
    load_color_slots<S>(B, n, k, n_views, a, s, b);
    float out[3][S], kappa[3];
    int status[3];
    qr_color_solve<S, float>(a, s, b, n_views, mu0, tries, trust, 7u, out, status, kappa);
    unsigned redo = 0u;
    if (prec != 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (status[c] == 1 || (status[c] == 0 && kappa[c] > 1e6f)) redo |= 1u << c;
        flags[k] = (uint8_t)redo;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (status[c] == 1 && !(redo & (1u << c)) && nfail) atomicAdd(nfail, 1);
#pragma unroll
        for (int i = 0; i < S; ++i) step[(size_t)(c * S + i) * n + k] = out[c][i];
    }
}

template <int S>
__global__ void __launch_bounds__(64) k_solve_color_qr64(DevScene sc, const float *__restrict__ B, int n_views,
                                                         float mu0, int tries, float trust, float *step,
                                                         int32_t *nfail, const uint8_t *__restrict__ flags,
                                                         unsigned long long *resolves, const float *__restrict__ rho) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = sc.n;
    if (k >= n) return;
    const unsigned redo = flags[k];
    if (!redo) return;
    if (rho) mu0 *= rho[k];   // learned per-Gaussian damping multiplier
    float a[QR_VMAX][3], s[QR_VMAX][3], b[QR_VMAX][S];
    load_color_slots<S>(B, n, k, n_views, a, s, b);
    float out[3][S], kappa[3];
    int status[3];
    qr_color_solve<S, double>(a, s, b, n_views, mu0, tries, trust, redo, out, status, kappa);
    if (resolves) atomicAdd(resolves, (unsigned long long)__popc(redo));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (!(redo & (1u << c))) continue;
        if (status[c] == 1 && nfail) atomicAdd(nfail, 1);
#pragma unroll
        for (int i = 0; i < S; ++i) step[(size_t)(c * S + i) * n + k] = out[c][i];
    }
}

// First-order baseline on the same blocks: step = -lr g (opacity: g plus the
// barrier's gradient), inside the Newton step's trust radii and bounds
// (position as a full 3D step; colour's gradient sum_v a_v b_v rebuilt from
// the per-view slots).  No contributing pixel (g and H zero): no step.
__global__ void k_solve_gradient(int group, DevScene sc, const float *__restrict__ B, int n_views, float lr,
                                 gs2_config cfg, float *step) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = sc.n, S = sc.S;
    if (k >= n) return;
    if (group == GS2_COLOR) {
        const size_t slot = (size_t)(6 + S) * n;
        for (int ch = 0; ch < 3; ++ch) {
            float x[GS2_MAX_SH];
            for (int i = 0; i < S; ++i) x[i] = 0.f;
            for (int v = 0; v < n_views; ++v) {
                const float *Bv = B + v * slot;
                const float a = Bv[(size_t)ch * n + k];
                if (a == 0.f) continue;
                for (int i = 0; i < S; ++i) x[i] -= lr * a * Bv[(size_t)(6 + i) * n + k];
            }
            trust_scale(S, x, cfg.trust_color);
            for (int i = 0; i < S; ++i) step[(size_t)(ch * S + i) * n + k] = x[i];
        }
        return;
    }
    const int D = (group == GS2_POS || group == GS2_SCALE) ? 3 : 1, NH = D * (D + 1) / 2;
    bool none = true;
    for (int i = 0; i < D + NH; ++i) none = none && B[(size_t)i * n + k] == 0.f;
    for (int i = 0; i < D; ++i) step[(size_t)i * n + k] = 0.f;
    if (none) return;
    if (group == GS2_POS) {
        float x[3];
        for (int i = 0; i < 3; ++i) x[i] = -lr * B[(size_t)i * n + k];
        const float smax = fmaxf(sc.scale[k], fmaxf(sc.scale[n + k], sc.scale[2 * n + k]));
        trust_scale(3, x, cfg.trust_pos * smax);
        for (int i = 0; i < 3; ++i) step[(size_t)i * n + k] = x[i];
    } else if (group == GS2_ROT) {
        float x = -lr * B[k];
        trust_scale(1, &x, cfg.trust_rot);
        step[k] = x;
    } else if (group == GS2_SCALE) {
        for (int i = 0; i < 3; ++i) {
            const float si = sc.scale[(size_t)i * n + k];
            const float ds = -lr * B[(size_t)i * n + k];
            step[(size_t)i * n + k] = fminf(fmaxf(ds, si / cfg.scale_trust - si), si * cfg.scale_trust - si);
        }
    } else {
        const float sg = sc.opacity[k], tau = cfg.frac_to_boundary;
        const float g = B[k] + cfg.barrier_alpha * (-1.f / sg + 1.f / (1.f - sg));
        step[k] = fminf(fmaxf(-lr * g, -tau * sg), tau * (1.f - sg));
    }
}

cudaError_t launch_solve(int group, const void *blocks, int n_views, const DevScene &sc, const DevCam &primary,
                         const gs2_config &cfg, void *step, int32_t *n_failed, uint8_t *flags, cudaStream_t st,
                         unsigned long long *resolves, const float *rho) {
    unsigned long long *rs = resolves ? resolves + group : nullptr;
    const int n = sc.n;
    if (n == 0) return cudaSuccess;
    const float *B = (const float *)blocks;
    float *s = (float *)step;
    const int g = (n + 255) / 256;
    if (cfg.gd_lr[group] > 0.f) {
        k_solve_gradient<<<g, 256, 0, st>>>(group, sc, B, n_views, cfg.gd_lr[group], cfg, s);
        GS2_COUNT_LAUNCH(1);
        return cudaGetLastError();
    }
    switch (group) {
    case GS2_POS:
        k_solve_pos<<<g, 256, 0, st>>>(sc, primary, B, cfg.damping_mu0, cfg.damping_tries, cfg.trust_pos, s,
                                       n_failed, cfg.precision, rs, rho);
        break;
    case GS2_ROT:
        k_solve_scalar<<<g, 256, 0, st>>>(n, B, cfg.damping_mu0, cfg.damping_tries, cfg.trust_rot, s, n_failed,
                                          cfg.precision, rs);
        break;
    case GS2_SCALE:
        k_solve_scale<<<g, 256, 0, st>>>(sc, primary, B, cfg.damping_mu0, cfg.damping_tries, cfg.near_z,
                                         cfg.scale_trust, s, n_failed, cfg.precision, rs, rho);
        break;
    case GS2_OPACITY:
        k_solve_opacity<<<g, 256, 0, st>>>(sc, B, cfg.damping_mu0, cfg.damping_tries, cfg.barrier_alpha,
                                           cfg.frac_to_boundary, s, n_failed, cfg.precision, rs);
        break;
    default:
        if (n_views <= 4) {
            const int gq = (n + 127) / 128;
            const int prec = (cfg.precision != 0 && flags) ? 1 : 0;
#define QR(SS)                                                                                                    \
    do {                                                                                                          \
        k_solve_color_qr<SS><<<gq, 128, 0, st>>>(sc, B, n_views, cfg.damping_mu0, cfg.damping_tries,              \
                                                 cfg.trust_color, s, n_failed, prec, flags, rho);                 \
        if (prec)                                                                                                 \
            k_solve_color_qr64<SS><<<(n + 63) / 64, 64, 0, st>>>(sc, B, n_views, cfg.damping_mu0,                 \
                                                                 cfg.damping_tries, cfg.trust_color, s, n_failed, \
                                                                 flags, rs, rho);                                 \
    } while (0)
            switch (sc.S) {
            case 1: QR(1); break;
            case 4: QR(4); break;
            case 9: QR(9); break;
            default: QR(16); break;
            }
#undef QR
        } else {
            k_solve_color<<<(3 * n + 127) / 128, 128, 0, st>>>(sc, B, n_views, cfg.damping_mu0, cfg.damping_tries,
                                                              cfg.trust_color, s, n_failed, cfg.precision, rs, rho);
        }
    }
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ apply
__global__ void k_apply(int group, DevScene sc, DevCam pr, const float *__restrict__ step, float scale_min) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = sc.n;
    if (k >= n) return;
    float *mean = const_cast<float *>(sc.mean), *quat = const_cast<float *>(sc.quat);
    float *scale = const_cast<float *>(sc.scale), *op = const_cast<float *>(sc.opacity);
    float *sh = const_cast<float *>(sc.sh);
    if (group == GS2_POS) {
        for (int i = 0; i < 3; ++i) mean[(size_t)i * n + k] += step[(size_t)i * n + k];
    } else if (group == GS2_ROT) {
        const float p[3] = {mean[k], mean[n + k], mean[2 * n + k]};
        float a[3];
        unit_dir(pr, p, a);
        const float th = step[k];
        const float cw = cosf(0.5f * th), sw = sinf(0.5f * th);
        const float q0 = quat[k], q1 = quat[n + k], q2 = quat[2 * n + k], q3 = quat[3 * n + k];
        const float adv = a[0] * q1 + a[1] * q2 + a[2] * q3;
        const float axv[3] = {a[1] * q3 - a[2] * q2, a[2] * q1 - a[0] * q3, a[0] * q2 - a[1] * q1};
        float qn[4];
        qn[0] = cw * q0 - sw * adv;
        qn[1] = cw * q1 + sw * (q0 * a[0] + axv[0]);
        qn[2] = cw * q2 + sw * (q0 * a[1] + axv[1]);
        qn[3] = cw * q3 + sw * (q0 * a[2] + axv[2]);
        const float in = rsqrtf(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
        for (int i = 0; i < 4; ++i) quat[(size_t)i * n + k] = qn[i] * in;
    } else if (group == GS2_SCALE) {
        for (int i = 0; i < 3; ++i) scale[(size_t)i * n + k] = fmaxf(scale[(size_t)i * n + k] + step[(size_t)i * n + k], scale_min);
    } else if (group == GS2_OPACITY) {
        op[k] += step[k];
    } else {
        for (int i = 0; i < 3 * sc.S; ++i) sh[(size_t)i * n + k] += step[(size_t)i * n + k];
    }
}

cudaError_t launch_apply(int group, const void *step, const DevScene &sc, const DevCam &primary,
                         const gs2_config &cfg, cudaStream_t st) {
    if (sc.n == 0) return cudaSuccess;
    k_apply<<<(sc.n + 255) / 256, 256, 0, st>>>(group, sc, primary, (const float *)step, cfg.scale_min);
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError();
}
