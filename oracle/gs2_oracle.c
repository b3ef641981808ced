/*
 * gs2 FP64 CPU ORACLE — TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * legs may load this library.  It shares no code, header, table or helper with
 * the CUDA path; it is the plain, slow, obviously-correct definition that the
 * GPU kernels are checked against.
 *
 * What it computes (paper section / equation in brackets):
 *   - projection of a 3D Gaussian: centre pi, EWA screen covariance Sigma,
 *     view direction r and SH colour c~              [Sec. 3, App. A.1-A.3]
 *   - brute-force per-pixel front-to-back compositing over ALL Gaussians in
 *     global depth order, no tiling                  [Eq. 3dgs]
 *   - per-pixel loss derivatives e = dL/dc, h = diag d2L/dc2 of
 *     L = L2 + lambda * L_SSIM                         [Sec. 4.2, loss eqs.]
 *   - per-Gaussian, per-group gradient and Hessian blocks by the chain rule
 *     of Eq. local_hessian_gradient, with dc/dy and d2c/dy2 obtained by
 *     second-order forward-mode jets (jet.h), i.e. exact derivatives of the
 *     compositing formula itself                        [Eq. local_hessian_gradient]
 *   - per-group damped local Newton solves and updates [Eq. local_newton,
 *     position / scaling / rotation / opacity / colour solves of Sec. 4.2]
 *   - camera KNN on the bounding sphere and the sweep with secondary targets
 *     [Sec. 4.1, Sec. 4.3 Eq. tildel]
 *
 * Readings of passages that are silent or garbled in the paper are listed at
 * each function; the same readings are implemented independently on the GPU.
 *
 * Parity pins: every function here is pinned by CPU tests against finite
 * differences, closed forms, invariants or textbook routines (tests/).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "jet.h"

int JD = 0;

enum { G_POS = 0, G_ROT = 1, G_SCALE = 2, G_OPACITY = 3, G_COLOR = 4, G_VALUES = -1 };

typedef struct {
    int n, sh_degree;
    double *mean;    /* [3][n] */
    double *quat;    /* [4][n] w,x,y,z */
    double *scale;   /* [3][n] linear scales */
    double *opacity; /* [n] in (0,1) */
    double *sh;      /* [3][S][n] channel-major */
} orc_scene;

typedef struct {
    int width, height;
    double fx, fy, cx, cy;
    double viewmat[12]; /* row-major [R | t], world -> camera; camera looks along +z */
    double clip_x, clip_y; /* frustum clamp of tx/tz, ty/tz in J; 0: 1.3 (W/2)/fx, 1.3 (H/2)/fy */
} orc_camera;

/* Frustum clamp limits of the projection Jacobian (reading: the standard 3DGS
 * rasteriser the paper builds on clamps tx/tz, ty/tz to 1.3x the half field of
 * view inside J; without it, Gaussians close to the camera plane and far off
 * axis become screen-space needles no FP32 rasteriser can evaluate). */
static double clip_lim(const orc_camera *c, int axis) {
    double v = axis == 0 ? c->clip_x : c->clip_y;
    if (v > 0) return v;
    return axis == 0 ? (double)(float)(1.3f * (0.5f * (float)c->width) / (float)c->fx)
                     : (double)(float)(1.3f * (0.5f * (float)c->height) / (float)c->fy);
}

typedef struct {
    double lambda_ssim;
    double alpha_min, alpha_max, t_min;
    double lowpass, near_z;
    double barrier_alpha, frac_to_boundary;
    double damping_mu0;
    int damping_tries;
    double scale_min;
    double ssim_c1, ssim_c2, ssim_sigma;
    int ssim_radius;
    int knn_k;
    int downsample;
    double scale_trust;
    double trust_pos;   /* |dp| <= trust_pos * max(s) */
    double trust_rot;   /* |theta| <= trust_rot */
    double trust_color; /* |dc_ch| <= trust_color (SH coefficient norm per channel) */
    int gauss_newton;   /* 1: drop the e d2c/dy2 term of the blocks (Gauss-Newton) */
    int group_order[5]; /* the groups of a sweep in the order run (a permutation of 0..4) */
    int group_jacobi;   /* 1: one render per view and sweep; every group solved at that state,
                           the steps applied together (position last) */
    double gd_lr[5];    /* > 0: that group takes the gradient step -gd_lr g instead of Newton's */
} orc_config;

/* Trust radii (reading; the paper fixes step size 1 and gives no safeguard):
 * a Jacobi step of a Gaussian seen by a handful of pixels is exact for its own
 * footprint but can be arbitrarily large; the step is scaled down to the
 * radius when it exceeds it, keeping its direction.  Non-finite steps become
 * zero and count as failed. */
static int trust_scale(int N, double *x, double radius) {
    double nn = 0;
    for (int i = 0; i < N; ++i) nn += x[i] * x[i];
    nn = sqrt(nn);
    if (!(nn == nn) || isinf(nn)) {
        for (int i = 0; i < N; ++i) x[i] = 0.0;
        return 1;
    }
    if (nn > radius) for (int i = 0; i < N; ++i) x[i] *= radius / nn;
    return 0;
}

int orc_sh_count(int degree) { return (degree + 1) * (degree + 1); }

/* ---------------------------------------------------------------------------
 * Real spherical-harmonic basis B_i * Phi_i(r), degrees 0..3  [App. A.2].
 * Phi is the paper's polynomial list; B are the orthonormal real-SH
 * normalisation constants sqrt((2l+1)/(4 pi) * (l-|m|)!/(l+|m|)! * (2 - delta_m0))
 * evaluated in closed form below, with the sign convention of the standard
 * 3DGS colour model (reading: the paper says it follows that pipeline).
 * ------------------------------------------------------------------------- */
static double SHB[16];
static int sh_init_done = 0;

static void sh_init(void) {
    if (sh_init_done) return;
    const double pi = 3.14159265358979323846;
    SHB[0] = sqrt(1.0 / (4.0 * pi));
    SHB[1] = sqrt(3.0 / (4.0 * pi));   /* Phi = -y */
    SHB[2] = sqrt(3.0 / (4.0 * pi));   /* Phi =  z */
    SHB[3] = sqrt(3.0 / (4.0 * pi));   /* Phi = -x */
    SHB[4] = sqrt(15.0 / (4.0 * pi));  /* xy */
    SHB[5] = -sqrt(15.0 / (4.0 * pi)); /* yz */
    SHB[6] = sqrt(5.0 / (16.0 * pi));  /* 2z^2 - x^2 - y^2 */
    SHB[7] = -sqrt(15.0 / (4.0 * pi)); /* xz */
    SHB[8] = sqrt(15.0 / (16.0 * pi)); /* x^2 - y^2 */
    SHB[9] = -sqrt(35.0 / (32.0 * pi));  /* y(3x^2 - y^2) */
    SHB[10] = sqrt(105.0 / (4.0 * pi));  /* xyz */
    SHB[11] = -sqrt(21.0 / (32.0 * pi)); /* y(4z^2 - x^2 - y^2) */
    SHB[12] = sqrt(7.0 / (16.0 * pi));   /* z(2z^2 - 3x^2 - 3y^2) */
    SHB[13] = -sqrt(21.0 / (32.0 * pi)); /* x(4z^2 - x^2 - y^2) */
    SHB[14] = sqrt(105.0 / (16.0 * pi)); /* z(x^2 - y^2) */
    SHB[15] = -sqrt(35.0 / (32.0 * pi)); /* x(x^2 - 3y^2) */
    sh_init_done = 1;
}

/* Phi_i(r) as jets, i < S; the paper's ordering (App. A.2). */
static void sh_phi_jet(int S, const jet r[3], jet *phi) {
    const jet *x = &r[0], *y = &r[1], *z = &r[2];
    jconst(&phi[0], 1.0);
    if (S <= 1) return;
    jscale(&phi[1], y, -1.0);
    jcopy(&phi[2], z);
    jscale(&phi[3], x, -1.0);
    if (S <= 4) return;
    jet xx, yy, zz, t1, t2;
    jmul(&xx, x, x);
    jmul(&yy, y, y);
    jmul(&zz, z, z);
    jmul(&phi[4], x, y);
    jmul(&phi[5], y, z);
    jscale(&t1, &zz, 2.0);
    jsub(&t1, &t1, &xx);
    jsub(&phi[6], &t1, &yy);
    jmul(&phi[7], x, z);
    jsub(&phi[8], &xx, &yy);
    if (S <= 9) return;
    /* y(3x^2 - y^2) */
    jscale(&t1, &xx, 3.0);
    jsub(&t1, &t1, &yy);
    jmul(&phi[9], y, &t1);
    /* xyz */
    jmul(&t1, x, y);
    jmul(&phi[10], &t1, z);
    /* y(4z^2 - x^2 - y^2) */
    jscale(&t1, &zz, 4.0);
    jsub(&t1, &t1, &xx);
    jsub(&t1, &t1, &yy);
    jmul(&phi[11], y, &t1);
    /* z(2z^2 - 3x^2 - 3y^2) */
    jscale(&t1, &zz, 2.0);
    jscale(&t2, &xx, 3.0);
    jsub(&t1, &t1, &t2);
    jscale(&t2, &yy, 3.0);
    jsub(&t1, &t1, &t2);
    jmul(&phi[12], z, &t1);
    /* x(4z^2 - x^2 - y^2) */
    jscale(&t1, &zz, 4.0);
    jsub(&t1, &t1, &xx);
    jsub(&t1, &t1, &yy);
    jmul(&phi[13], x, &t1);
    /* z(x^2 - y^2) */
    jsub(&t1, &xx, &yy);
    jmul(&phi[14], z, &t1);
    /* x(x^2 - 3y^2) */
    jscale(&t2, &yy, 3.0);
    jsub(&t1, &xx, &t2);
    jmul(&phi[15], x, &t1);
}

/* Exported: B_i Phi_i(r) for a plain direction (used by the orthonormality pin). */
void orc_sh_basis(double x, double y, double z, int degree, double *out) {
    sh_init();
    int save = JD;
    JD = 0;
    int S = orc_sh_count(degree);
    jet r[3], phi[16];
    jconst(&r[0], x);
    jconst(&r[1], y);
    jconst(&r[2], z);
    sh_phi_jet(S, r, phi);
    for (int i = 0; i < S; ++i) out[i] = SHB[i] * phi[i].v;
    JD = save;
}

/* camera centre o = -R^T t */
static void cam_center(const orc_camera *c, double o[3]) {
    const double *V = c->viewmat;
    for (int i = 0; i < 3; ++i) o[i] = -(V[0 * 4 + i] * V[3] + V[1 * 4 + i] * V[7] + V[2 * 4 + i] * V[11]);
}

/* Depth key: camera-space z in FP64, summed in this fixed order, rounded to
 * FP32.  Products of FP32-representable inputs are exact in FP64, so any
 * implementation that sums in this order obtains the same key bit for bit
 * (reading of "sorted based on depth" [Sec. 3]: order = (key, index)). */
static double depth_fp64(const orc_camera *c, double px, double py, double pz) {
    const double *V = c->viewmat;
    double a = V[8] * px;
    a = a + V[9] * py;
    a = a + V[10] * pz;
    a = a + V[11];
    return a;
}

/* ---------------------------------------------------------------------------
 * Parameters of Gaussian k as jets; the free variables depend on the group:
 *   POS: p (3)   ROT: theta (1) about axis   SCALE: s (3)   OPACITY: sigma (1)
 *   COLOR: the S SH coefficients of channel ch     VALUES: none (JD = 0)
 * Rotation reading [Sec. 4.2 rotation solve]: dq = (cos(theta/2), sin(theta/2) a)
 * with a the unit camera->centre direction of the primary view, applied as
 * q <- dq (x) q (Hamilton product).
 * ------------------------------------------------------------------------- */
typedef struct {
    jet p[3], q[4], s[3], op;
    jet sh[3][16];
} gparams;

static void load_params(const orc_scene *sc, int k, int group, int ch, const double axis[3], gparams *P) {
    int n = sc->n, S = orc_sh_count(sc->sh_degree);
    for (int i = 0; i < 3; ++i) {
        if (group == G_POS) jvar(&P->p[i], sc->mean[i * n + k], i);
        else jconst(&P->p[i], sc->mean[i * n + k]);
        if (group == G_SCALE) jvar(&P->s[i], sc->scale[i * n + k], i);
        else jconst(&P->s[i], sc->scale[i * n + k]);
    }
    if (group == G_OPACITY) jvar(&P->op, sc->opacity[k], 0);
    else jconst(&P->op, sc->opacity[k]);
    for (int c = 0; c < 3; ++c)
        for (int i = 0; i < S; ++i) {
            double v = sc->sh[(c * S + i) * n + k];
            if (group == G_COLOR && c == ch) jvar(&P->sh[c][i], v, i);
            else jconst(&P->sh[c][i], v);
        }
    if (group == G_ROT) {
        jet th, half, cw, sw;
        jvar(&th, 0.0, 0);
        jscale(&half, &th, 0.5);
        jcos(&cw, &half);
        jsin(&sw, &half);
        double q0[4];
        for (int i = 0; i < 4; ++i) q0[i] = sc->quat[i * n + k];
        /* dq = (cw, sw*a); q' = dq (x) q0 :
         *   w' = cw*w0 - sw*(a . v0)
         *   v' = cw*v0 + w0*sw*a + sw*(a x v0)                                 */
        double adotv = axis[0] * q0[1] + axis[1] * q0[2] + axis[2] * q0[3];
        double axv[3] = {axis[1] * q0[3] - axis[2] * q0[2], axis[2] * q0[1] - axis[0] * q0[3],
                         axis[0] * q0[2] - axis[1] * q0[1]};
        jet t;
        jscale(&P->q[0], &cw, q0[0]);
        jscale(&t, &sw, -adotv);
        jadd(&P->q[0], &P->q[0], &t);
        for (int i = 0; i < 3; ++i) {
            jscale(&P->q[1 + i], &cw, q0[1 + i]);
            jscale(&t, &sw, q0[0] * axis[i] + axv[i]);
            jadd(&P->q[1 + i], &P->q[1 + i], &t);
        }
    } else {
        for (int i = 0; i < 4; ++i) jconst(&P->q[i], sc->quat[i * n + k]);
    }
}

/* Projection result of one Gaussian in one view (jets). */
typedef struct {
    int culled;
    double tz;
    float key;
    jet pix[2];   /* pi: pixel coordinates of the centre */
    jet sig[3];   /* Sigma2D (xx, xy, yy) incl. low-pass */
    jet con[3];   /* conic = Sigma2D^{-1} (xx, xy, yy) */
    jet op;       /* sigma */
    jet col[3];   /* view-dependent colour c~ */
} gproj;

/* Rotation matrix of a (normalised) quaternion w,x,y,z. */
static void quat_to_R(const jet q[4], jet R[3][3]) {
    jet n2, t, nrm, qn[4];
    jmul(&n2, &q[0], &q[0]);
    for (int i = 1; i < 4; ++i) {
        jmul(&t, &q[i], &q[i]);
        jadd(&n2, &n2, &t);
    }
    jsqrt(&nrm, &n2);
    for (int i = 0; i < 4; ++i) jdiv(&qn[i], &q[i], &nrm);
    const jet *w = &qn[0], *x = &qn[1], *y = &qn[2], *z = &qn[3];
    jet xx, yy, zz, xy, xz, yz, wx, wy, wz;
    jmul(&xx, x, x); jmul(&yy, y, y); jmul(&zz, z, z);
    jmul(&xy, x, y); jmul(&xz, x, z); jmul(&yz, y, z);
    jmul(&wx, w, x); jmul(&wy, w, y); jmul(&wz, w, z);
    jet s;
    jadd(&s, &yy, &zz); jscale(&s, &s, -2.0); jaddc(&R[0][0], &s, 1.0);
    jsub(&s, &xy, &wz); jscale(&R[0][1], &s, 2.0);
    jadd(&s, &xz, &wy); jscale(&R[0][2], &s, 2.0);
    jadd(&s, &xy, &wz); jscale(&R[1][0], &s, 2.0);
    jadd(&s, &xx, &zz); jscale(&s, &s, -2.0); jaddc(&R[1][1], &s, 1.0);
    jsub(&s, &yz, &wx); jscale(&R[1][2], &s, 2.0);
    jsub(&s, &xz, &wy); jscale(&R[2][0], &s, 2.0);
    jadd(&s, &yz, &wx); jscale(&R[2][1], &s, 2.0);
    jadd(&s, &xx, &yy); jscale(&s, &s, -2.0); jaddc(&R[2][2], &s, 1.0);
}

/* ---------------------------------------------------------------------------
 * Projection [Sec. 3, App. A.1, A.3]; readings:
 *  - pinhole camera looking along +z (x right, y down): the paper's
 *    pi = (W/2) h_x/h_w + const with h = P W [p;1] is this map for the
 *    projection matrix P with h_w = t_z; pi = (fx tx/tz + cx, fy ty/tz + cy),
 *    pixel (m, n) has its centre at integer coordinates (m, n);
 *  - EWA: Sigma2D = J Wr R S S^T R^T Wr^T J^T + lowpass*I with J the
 *    perspective Jacobian at t (the paper's "orthographic" is read as the
 *    Jacobian of the projection P), with tx/tz, ty/tz clamped to the frustum
 *    limits inside J (the standard 3DGS clamp; clip_lim);
 *  - a Gaussian with t_z < near_z is culled;
 *  - c~ = sum_i B_i Phi_i(r) c_i with r the unit camera->centre direction, no
 *    offset and no clamp (c~ is linear in c, as the colour solve states).
 * ------------------------------------------------------------------------- */
static void project_one(const orc_camera *cam, const orc_config *cfg, int S, gparams *P, gproj *out) {
    const double *V = cam->viewmat;
    out->tz = depth_fp64(cam, P->p[0].v, P->p[1].v, P->p[2].v);
    out->key = (float)out->tz;
    out->culled = !(out->tz >= cfg->near_z);
    if (out->culled) return;

    jet t[3], tmp;
    for (int i = 0; i < 3; ++i) {
        jscale(&t[i], &P->p[0], V[i * 4 + 0]);
        jaxpy(&t[i], V[i * 4 + 1], &P->p[1]);
        jaxpy(&t[i], V[i * 4 + 2], &P->p[2]);
        jaddc(&t[i], &t[i], V[i * 4 + 3]);
    }
    jet itz, itz2;
    jrecip(&itz, &t[2]);
    jmul(&itz2, &itz, &itz);
    /* pi */
    jmul(&tmp, &t[0], &itz);
    jscale(&tmp, &tmp, cam->fx);
    jaddc(&out->pix[0], &tmp, cam->cx);
    jmul(&tmp, &t[1], &itz);
    jscale(&tmp, &tmp, cam->fy);
    jaddc(&out->pix[1], &tmp, cam->cy);

    /* J (2x3) with tau = t_xy / t_z clamped to the frustum limits (a clamped
     * tau is a constant) */
    jet J[2][3], tau[2];
    for (int a = 0; a < 2; ++a) {
        double L = clip_lim(cam, a);
        jmul(&tau[a], &t[a], &itz);
        if (tau[a].v > L) jconst(&tau[a], L);
        else if (tau[a].v < -L) jconst(&tau[a], -L);
    }
    jscale(&J[0][0], &itz, cam->fx);
    jconst(&J[0][1], 0.0);
    jmul(&tmp, &tau[0], &itz);
    jscale(&J[0][2], &tmp, -cam->fx);
    jconst(&J[1][0], 0.0);
    jscale(&J[1][1], &itz, cam->fy);
    jmul(&tmp, &tau[1], &itz);
    jscale(&J[1][2], &tmp, -cam->fy);

    /* M = J Wr R diag(s)  (2x3); Sigma2D = M M^T + lowpass I */
    jet R[3][3], JW[2][3], JWR[2][3], M[2][3];
    quat_to_R(P->q, R);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b) {
            jscale(&JW[a][b], &J[a][0], V[0 * 4 + b]);
            jaxpy(&JW[a][b], V[1 * 4 + b], &J[a][1]);
            jaxpy(&JW[a][b], V[2 * 4 + b], &J[a][2]);
        }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b) {
            jmul(&JWR[a][b], &JW[a][0], &R[0][b]);
            jmul(&tmp, &JW[a][1], &R[1][b]);
            jadd(&JWR[a][b], &JWR[a][b], &tmp);
            jmul(&tmp, &JW[a][2], &R[2][b]);
            jadd(&JWR[a][b], &JWR[a][b], &tmp);
            jmul(&M[a][b], &JWR[a][b], &P->s[b]);
        }
    int idx[3][2] = {{0, 0}, {0, 1}, {1, 1}};
    for (int e = 0; e < 3; ++e) {
        int a = idx[e][0], b = idx[e][1];
        jmul(&out->sig[e], &M[a][0], &M[b][0]);
        jmul(&tmp, &M[a][1], &M[b][1]);
        jadd(&out->sig[e], &out->sig[e], &tmp);
        jmul(&tmp, &M[a][2], &M[b][2]);
        jadd(&out->sig[e], &out->sig[e], &tmp);
    }
    jaddc(&out->sig[0], &out->sig[0], cfg->lowpass);
    jaddc(&out->sig[2], &out->sig[2], cfg->lowpass);
    /* conic */
    jet det, idet;
    jmul(&det, &out->sig[0], &out->sig[2]);
    jmul(&tmp, &out->sig[1], &out->sig[1]);
    jsub(&det, &det, &tmp);
    jrecip(&idet, &det);
    jmul(&out->con[0], &out->sig[2], &idet);
    jmul(&out->con[1], &out->sig[1], &idet);
    jscale(&out->con[1], &out->con[1], -1.0);
    jmul(&out->con[2], &out->sig[0], &idet);

    jcopy(&out->op, &P->op);

    /* view direction and SH colour */
    double o[3];
    cam_center(cam, o);
    jet d[3], d2, rho, r[3], phi[16];
    for (int i = 0; i < 3; ++i) jaddc(&d[i], &P->p[i], -o[i]);
    jmul(&d2, &d[0], &d[0]);
    jmul(&tmp, &d[1], &d[1]);
    jadd(&d2, &d2, &tmp);
    jmul(&tmp, &d[2], &d[2]);
    jadd(&d2, &d2, &tmp);
    jsqrt(&rho, &d2);
    for (int i = 0; i < 3; ++i) jdiv(&r[i], &d[i], &rho);
    sh_phi_jet(S, r, phi);
    for (int c = 0; c < 3; ++c) {
        jconst(&out->col[c], 0.0);
        for (int i = 0; i < S; ++i) {
            jmul(&tmp, &phi[i], &P->sh[c][i]);
            jaxpy(&out->col[c], SHB[i], &tmp);
        }
    }
}

/* ---------------------------------------------------------------------------
 * FP32 decisions [Sec. 3, Eq. 3dgs].  Three outcomes of the forward pass are
 * discrete: whether a (pixel, Gaussian) term is composited (sigma G >=
 * alpha_min), whether its alpha is clamped (sigma G > alpha_max), and which
 * screen tiles list the Gaussian.  Floating point decides them, so (reading)
 * they are taken in the kernel's precision: FP32, from the FP32 parameters and
 * camera, with correctly rounded operations only (+, -, *, fma, /, sqrt;
 * floor, ceil, min, max are exact) in the order written below, and a
 * logarithm taken by the atanh (Gregory) series instead of a library call.
 * Every IEEE FP32 evaluation of these steps gives the same bits.  In terms of
 * the quadratic form q = d^T Sigma^-1 d of the pixel offset d:
 *   composited <=> q <= l = 2 ln(sigma / alpha_min),
 *   clamped    <=> q <  lmax = 2 ln(sigma / alpha_max) (-1 if sigma <= alpha_max),
 * the same sets as in exact arithmetic.  Everything the oracle computes with
 * those decisions (alpha, T, colours, derivatives) stays FP64.  The oracle
 * file is compiled with -ffp-contract=off, so a * b + c below is two rounded
 * operations and fmaf is one.
 * ------------------------------------------------------------------------- */
typedef struct {
    float px, py, ca, cb, cc, sxx, syy, k2, l, lmax, rx, ry;
    unsigned rect_lo, rect_hi; /* tile box: tx0 | ty0 << 16, tx1 | ty1 << 16 (exclusive ends) */
    unsigned touched;          /* tiles of the box */
} dec32;

/* ln x for finite x >= 1: x = 2^e m with m in [sqrt(1/2), sqrt(2)],
 * ln m = 2 atanh(u) = 2 u (1 + u^2/3 + u^4/5 + u^6/7 + u^8/9), u = (m-1)/(m+1). */
static float d_ln(float x) {
    int e = 0;
    float m = frexpf(x, &e); /* x = m 2^e, m in [1/2, 1) */
    m = m * 2.0f;
    e -= 1;
    if (m > 0x1.6a09e6p+0f) {
        m = m * 0.5f;
        e += 1;
    }
    float u = (m - 1.0f) / (m + 1.0f);
    float s = u * u;
    float p = 0x1.c71c72p-4f;
    p = fmaf(p, s, 0x1.24924ap-3f);
    p = fmaf(p, s, 0x1.99999ap-3f);
    p = fmaf(p, s, 0x1.555556p-2f);
    p = fmaf(p, s, 1.0f);
    float lm = (2.0f * u) * p;
    return fmaf((float)e, 0x1.62e430p-1f, lm);
}

/* q = dx (ca dx + 2 cb dy) + cc dy^2 as fma(dx, fma(cb, dy, fma(ca, dx, cb dy)), (cc dy) dy) */
static float d_quad(float ca, float cb, float cc, float dx, float dy) {
    float a = fmaf(ca, dx, cb * dy);
    a = fmaf(cb, dy, a);
    return fmaf(dx, a, (cc * dy) * dy);
}

static float fmin32(float a, float b) { return a < b ? a : b; }
static float fmax32(float a, float b) { return a > b ? a : b; }

/* The FP32 projection of one Gaussian in front of the camera (tz the FP32
 * depth key, sigma >= alpha_min): screen centre, EWA covariance and conic,
 * the thresholds, the padded support box and its tile rectangle. */
static void dec32_project(const orc_camera *cam, const orc_config *cfg, const float p[3], float tz, const float q[4],
                          const float sc[3], float sigma, int tile, dec32 *r) {
    float V[12];
    for (int i = 0; i < 12; ++i) V[i] = (float)cam->viewmat[i];
    const float fx = (float)cam->fx, fy = (float)cam->fy, cx = (float)cam->cx, cy = (float)cam->cy;
    const float Lx = (float)clip_lim(cam, 0), Ly = (float)clip_lim(cam, 1);
    const float lowpass = (float)cfg->lowpass, amin = (float)cfg->alpha_min, amax = (float)cfg->alpha_max;
    /* camera-space centre and the 2x3 T = J Wr */
    float tx = fmaf(V[0], p[0], fmaf(V[1], p[1], fmaf(V[2], p[2], V[3])));
    float ty = fmaf(V[4], p[0], fmaf(V[5], p[1], fmaf(V[6], p[2], V[7])));
    float itz = 1.0f / tz;
    float taux = fmin32(fmax32(tx * itz, -Lx), Lx);
    float tauy = fmin32(fmax32(ty * itz, -Ly), Ly);
    float j00 = fx * itz, j02 = ((-fx) * taux) * itz;
    float j11 = fy * itz, j12 = ((-fy) * tauy) * itz;
    float T0[3], T1[3];
    for (int j = 0; j < 3; ++j) {
        T0[j] = fmaf(j00, V[j], j02 * V[8 + j]);
        T1[j] = fmaf(j11, V[4 + j], j12 * V[8 + j]);
    }
    /* rotation of the normalised quaternion */
    float qq = fmaf(q[0], q[0], fmaf(q[1], q[1], fmaf(q[2], q[2], q[3] * q[3])));
    float qn = 1.0f / sqrtf(qq);
    float w = q[0] * qn, x = q[1] * qn, y = q[2] * qn, z = q[3] * qn;
    float R[3][3];
    R[0][0] = 1.0f - 2.0f * fmaf(y, y, z * z);
    R[0][1] = 2.0f * (x * y - w * z);
    R[0][2] = 2.0f * (x * z + w * y);
    R[1][0] = 2.0f * (x * y + w * z);
    R[1][1] = 1.0f - 2.0f * fmaf(x, x, z * z);
    R[1][2] = 2.0f * (y * z - w * x);
    R[2][0] = 2.0f * (x * z - w * y);
    R[2][1] = 2.0f * (y * z + w * x);
    R[2][2] = 1.0f - 2.0f * fmaf(x, x, y * y);
    /* Sigma2D = sum_j s_j^2 m_j m_j^T with m_j = T R e_j */
    float ss[3] = {sc[0] * sc[0], sc[1] * sc[1], sc[2] * sc[2]};
    float m0[3], m1[3], sxx = 0.0f, sxy = 0.0f, syy = 0.0f;
    for (int j = 0; j < 3; ++j) {
        m0[j] = fmaf(T0[0], R[0][j], fmaf(T0[1], R[1][j], T0[2] * R[2][j]));
        m1[j] = fmaf(T1[0], R[0][j], fmaf(T1[1], R[1][j], T1[2] * R[2][j]));
        float a0 = ss[j] * m0[j];
        sxx = fmaf(a0, m0[j], sxx);
        sxy = fmaf(a0, m1[j], sxy);
        syy = fmaf(ss[j] * m1[j], m1[j], syy);
    }
    /* det(A + l I) = det A + l tr A + l^2; det A by Cauchy-Binet */
    float detA = 0.0f;
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j) {
            float cr = fmaf(m0[i], m1[j], -(m1[i] * m0[j]));
            detA = fmaf((ss[i] * ss[j]) * cr, cr, detA);
        }
    float det = (detA + lowpass * (sxx + syy)) + lowpass * lowpass;
    sxx = sxx + lowpass;
    syy = syy + lowpass;
    float idet = 1.0f / det;
    r->ca = syy * idet;
    r->cb = (-sxy) * idet;
    r->cc = sxx * idet;
    r->sxx = sxx;
    r->syy = syy;
    r->k2 = det / (syy * syy);
    r->px = fmaf(fx * tx, itz, cx);
    r->py = fmaf(fy * ty, itz, cy);
    /* alpha_min = 0 (every threshold off, a setting of the smooth oracle pins
     * only; the library requires alpha_min > 0): every term is composited */
    r->l = amin > 0.0f ? 2.0f * d_ln(sigma / amin) : INFINITY;
    r->lmax = sigma > amax ? 2.0f * d_ln(sigma / amax) : -1.0f;
    r->rx = fmaf(sqrtf(fmax32(r->l * sxx, 0.0f)), 1.0005f, 0.02f);
    r->ry = fmaf(sqrtf(fmax32(r->l * syy, 0.0f)), 1.0005f, 0.02f);
    /* tile rectangle of the support box */
    float fx0 = fmax32(ceilf(r->px - r->rx), 0.0f), fx1 = fmin32(floorf(r->px + r->rx), (float)(cam->width - 1));
    float fy0 = fmax32(ceilf(r->py - r->ry), 0.0f), fy1 = fmin32(floorf(r->py + r->ry), (float)(cam->height - 1));
    r->rect_lo = r->rect_hi = 0u;
    r->touched = 0u;
    if (fx0 <= fx1 && fy0 <= fy1) {
        unsigned tx0 = (unsigned)fx0 / tile, tx1 = (unsigned)fx1 / tile + 1u;
        unsigned ty0 = (unsigned)fy0 / tile, ty1 = (unsigned)fy1 / tile + 1u;
        r->touched = (tx1 - tx0) * (ty1 - ty0);
        r->rect_lo = tx0 | (ty0 << 16);
        r->rect_hi = tx1 | (ty1 << 16);
    }
}

/* Does the support { q <= l } reach a pixel of the tile with columns
 * [x0, x0 + t) and rows [y0, y0 + t)?  Row by row (y relative to the centre)
 * the support is |x - k1 y| <= sqrt(k2 (ry^2 - y^2)), k1 = -cb / ca; over the
 * tile's rows the extreme x lie at the rows nearest +-y*, y* = k1 ry /
 * sqrt(k2 + k1^2); the reach is widened by 1e-3 (|k1| + sqrt(k2)) ry + 0.05 px. */
static int d_support_reaches(const dec32 *d, float x0, float y0, float t) {
    float k1 = (-d->cb) / d->ca;
    float ystar = (k1 * d->ry) / sqrtf(fmaf(k1, k1, d->k2));
    float marg = fmaf(1e-3f, (fabsf(k1) + sqrtf(d->k2)) * d->ry, 0.05f);
    float ylo = fmax32(y0, ceilf(d->py - d->ry));
    float yhi = fmin32((y0 + t) - 1.0f, floorf(d->py + d->ry));
    if (!(ylo <= yhi)) return 0;
    float ya = ylo - d->py, yb = yhi - d->py;
    float yr = fmin32(fmax32(ystar, ya), yb), yl = fmin32(fmax32(-ystar, ya), yb);
    float r2 = d->ry * d->ry;
    float hr = sqrtf(fmax32(d->k2 * (r2 - yr * yr), 0.0f));
    float hl = sqrtf(fmax32(d->k2 * (r2 - yl * yl), 0.0f));
    float xr = (fmaf(k1, yr, d->px) + hr) + marg;
    float xl = (fmaf(k1, yl, d->px) - hl) - marg;
    float c0 = fmax32(ceilf(xl), x0);
    float c1 = fmin32(floorf(xr), (x0 + t) - 1.0f);
    return c0 <= c1;
}

/* the decision record of Gaussian k from the scene's (FP32-valued) parameters */
static void dec32_of(const orc_scene *sc, const orc_camera *cam, const orc_config *cfg, int k, float tz, int tile,
                     dec32 *r) {
    int n = sc->n;
    float p[3], q[4], s3[3];
    for (int i = 0; i < 3; ++i) {
        p[i] = (float)sc->mean[i * n + k];
        s3[i] = (float)sc->scale[i * n + k];
    }
    for (int i = 0; i < 4; ++i) q[i] = (float)sc->quat[i * n + k];
    dec32_project(cam, cfg, p, tz, q, s3, (float)sc->opacity[k], tile, r);
}

/* ---------------------------------------------------------------------------
 * Per-view projected set, packed; plus the global depth order.
 * ------------------------------------------------------------------------- */
#define NPJ 9 /* packed jets: pix0 pix1 con0 con1 con2 op col0 col1 col2 */

typedef struct {
    int n;
    int js;          /* doubles per packed jet */
    double *jets;    /* [n][NPJ][js] */
    double *plain;   /* [n][NPJ] values */
    double *sig;     /* [n][3] Sigma2D values */
    double *tz;      /* [n] */
    float *key;      /* [n] */
    int *culled;     /* [n] */
    int *order;      /* sorted non-culled Gaussians with sigma >= alpha_min */
    int norder;
    dec32 *dec;      /* [n] FP32 decision records of the ordered Gaussians (16x16 tiles) */
} viewset;

static const float *g_sort_key;
static int cmp_order(const void *a, const void *b) {
    int i = *(const int *)a, j = *(const int *)b;
    float ki = g_sort_key[i], kj = g_sort_key[j];
    if (ki < kj) return -1;
    if (ki > kj) return 1;
    return (i < j) ? -1 : (i > j);
}

static void viewset_free(viewset *vs) {
    free(vs->jets); free(vs->plain); free(vs->sig); free(vs->tz); free(vs->key);
    free(vs->culled); free(vs->order); free(vs->dec);
}

/* Project every Gaussian with the variable assignment of (group, ch). */
static void viewset_build(viewset *vs, const orc_scene *sc, const orc_camera *cam, const orc_camera *primary,
                          const orc_config *cfg, int group, int ch) {
    sh_init();
    int n = sc->n, S = orc_sh_count(sc->sh_degree);
    vs->n = n;
    vs->js = jsize();
    vs->jets = (double *)malloc(sizeof(double) * (size_t)n * NPJ * vs->js);
    vs->plain = (double *)malloc(sizeof(double) * (size_t)n * NPJ);
    vs->sig = (double *)malloc(sizeof(double) * (size_t)n * 3);
    vs->tz = (double *)malloc(sizeof(double) * n);
    vs->key = (float *)malloc(sizeof(float) * n);
    vs->culled = (int *)malloc(sizeof(int) * n);
    vs->order = (int *)malloc(sizeof(int) * n);
    vs->dec = (dec32 *)calloc((size_t)n, sizeof(dec32));
    double o[3];
    cam_center(primary, o);
#pragma omp parallel for schedule(dynamic, 16)
    for (int k = 0; k < n; ++k) {
        double axis[3] = {0, 0, 1};
        if (group == G_ROT) {
            double d[3], nn = 0;
            for (int i = 0; i < 3; ++i) {
                d[i] = sc->mean[i * n + k] - o[i];
                nn += d[i] * d[i];
            }
            nn = sqrt(nn);
            for (int i = 0; i < 3; ++i) axis[i] = d[i] / nn;
        }
        gparams P;
        gproj G;
        load_params(sc, k, group, ch, axis, &P);
        project_one(cam, cfg, S, &P, &G);
        vs->tz[k] = G.tz;
        vs->key[k] = G.key;
        vs->culled[k] = G.culled;
        double *dst = vs->jets + (size_t)k * NPJ * vs->js;
        if (G.culled) {
            memset(dst, 0, sizeof(double) * NPJ * vs->js);
            for (int i = 0; i < NPJ; ++i) vs->plain[k * NPJ + i] = 0.0;
            for (int i = 0; i < 3; ++i) vs->sig[k * 3 + i] = 0.0;
            continue;
        }
        const jet *list[NPJ] = {&G.pix[0], &G.pix[1], &G.con[0], &G.con[1], &G.con[2],
                                &G.op, &G.col[0], &G.col[1], &G.col[2]};
        for (int i = 0; i < NPJ; ++i) {
            jpack(dst + i * vs->js, list[i]);
            vs->plain[k * NPJ + i] = list[i]->v;
        }
        for (int i = 0; i < 3; ++i) vs->sig[k * 3 + i] = G.sig[i].v;
    }
    int m = 0;
    for (int k = 0; k < n; ++k)
        if (!vs->culled[k] && vs->plain[k * NPJ + 5] >= cfg->alpha_min) vs->order[m++] = k;
    vs->norder = m;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i) dec32_of(sc, cam, cfg, vs->order[i], vs->key[vs->order[i]], 16, &vs->dec[vs->order[i]]);
    g_sort_key = vs->key;
    qsort(vs->order, m, sizeof(int), cmp_order);
}

/* ---------------------------------------------------------------------------
 * Compositing of one pixel [Eq. 3dgs], front to back over the global order.
 * Readings (standard 3DGS rasterisation constants, all config fields):
 *   alpha = min(sigma G, alpha_max); a term with alpha < alpha_min is skipped;
 *   compositing stops before the term that would take T below t_min;
 *   black background.
 * Whether a term is skipped or clamped is the FP32 decision of its record
 * (q <= l, q < lmax: see "FP32 decisions"); alpha, T and the colour are FP64.
 * Records every contributor (index, alpha, T before it) and the smallest
 * relative distance of the early-stop decision (the one decision still taken
 * in FP64 here) from its threshold.
 * ------------------------------------------------------------------------- */
typedef struct {
    int k;
    double alpha, T, G;
    int clamped;
} contrib;

static int pixel_pass(const viewset *vs, const orc_config *cfg, double px, double py, contrib *list,
                      double color[3], double *T_out, double *margin) {
    double T = 1.0, C[3] = {0, 0, 0}, mg = INFINITY;
    int nc = 0;
    for (int oi = 0; oi < vs->norder; ++oi) {
        int k = vs->order[oi];
        const double *pl = vs->plain + k * NPJ;
        const dec32 *D = vs->dec + k;
        float q32 = d_quad(D->ca, D->cb, D->cc, (float)px - D->px, (float)py - D->py);
        if (!(q32 <= D->l)) continue;  /* sigma G < alpha_min */
        int clamped = q32 < D->lmax;    /* sigma G > alpha_max */
        double dx = px - pl[0], dy = py - pl[1];
        double power = -0.5 * (pl[2] * dx * dx + 2.0 * pl[3] * dx * dy + pl[4] * dy * dy);
        double G = exp(power);
        double alpha = clamped ? cfg->alpha_max : pl[5] * G;
        double testT = T * (1.0 - alpha);
        if (cfg->t_min > 0) {
            double m3 = fabs(testT - cfg->t_min) / cfg->t_min;
            if (m3 < mg) mg = m3;
        }
        if (testT < cfg->t_min) break;
        for (int c = 0; c < 3; ++c) C[c] += alpha * T * pl[6 + c];
        if (list) {
            list[nc].k = k;
            list[nc].alpha = alpha;
            list[nc].T = T;
            list[nc].G = G;
            list[nc].clamped = clamped;
        }
        nc++;
        T = testT;
    }
    for (int c = 0; c < 3; ++c) color[c] = C[c];
    *T_out = T;
    if (margin) *margin = mg;
    return nc;
}

/* Exported: per-Gaussian projection values.
 * out [15][n]: pix_x pix_y sxx sxy syy con_xx con_xy con_yy sigma col0 col1 col2 tz culled (unused)
 * key [n] float. */
int orc_project(const orc_scene *sc, const orc_camera *cam, const orc_config *cfg, double *out, float *key) {
    int save = JD;
    JD = 0;
    viewset vs;
    viewset_build(&vs, sc, cam, cam, cfg, G_VALUES, 0);
    int n = sc->n;
    for (int k = 0; k < n; ++k) {
        const double *pl = vs.plain + k * NPJ;
        out[0 * n + k] = pl[0];
        out[1 * n + k] = pl[1];
        for (int i = 0; i < 3; ++i) out[(2 + i) * n + k] = vs.sig[k * 3 + i];
        for (int i = 0; i < 3; ++i) out[(5 + i) * n + k] = pl[2 + i];
        out[8 * n + k] = pl[5];
        for (int i = 0; i < 3; ++i) out[(9 + i) * n + k] = pl[6 + i];
        out[12 * n + k] = vs.tz[k];
        out[13 * n + k] = vs.culled[k];
        out[14 * n + k] = 0.0;
        key[k] = vs.key[k];
    }
    viewset_free(&vs);
    JD = save;
    return 0;
}

/* Exported: brute-force render.  image [3][H][W], tfinal [H][W], ncontrib [H][W],
 * margin [H][W] (smallest relative threshold distance seen at the pixel). */
int orc_render(const orc_scene *sc, const orc_camera *cam, const orc_config *cfg, double *image, double *tfinal,
               int *ncontrib, double *margin) {
    int save = JD;
    JD = 0;
    viewset vs;
    viewset_build(&vs, sc, cam, cam, cfg, G_VALUES, 0);
    int W = cam->width, H = cam->height;
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double C[3], T, mg;
            int nc = pixel_pass(&vs, cfg, (double)x, (double)y, NULL, C, &T, &mg);
            for (int c = 0; c < 3; ++c) image[(size_t)c * W * H + (size_t)y * W + x] = C[c];
            if (tfinal) tfinal[(size_t)y * W + x] = T;
            if (ncontrib) ncontrib[(size_t)y * W + x] = nc;
            if (margin) margin[(size_t)y * W + x] = mg;
        }
    viewset_free(&vs);
    JD = save;
    return 0;
}

/* ---------------------------------------------------------------------------
 * Loss and its per-pixel derivatives [Sec. 4.2, loss equations]. Readings:
 *   L2  = 1/(3|I|) sum_p sum_ch 1/2 (c - c^t)^2
 *   L_S = 1/(3|I|) sum_p sum_ch (1 - SSIM_ch(p))
 *   SSIM: Wang-2004 per channel with an 11x11 Gaussian window (sigma 1.5),
 *   zero-padded "same" windows, C1 = 0.01^2, C2 = 0.03^2 (the printed F_S
 *   denominator is garbled; the standard form is used);
 *   e = dL/dc exactly; h = d2L/dc2 on the pixel diagonal only, i.e. the exact
 *   second derivative wrt c_q of every window containing q, summed.
 * The derivative wrt one pixel value is taken with a one-variable
 * second-order jet through the window statistics.
 * ------------------------------------------------------------------------- */
typedef struct { double v, d, dd; } sj1;
static inline sj1 j1c(double v) { sj1 r = {v, 0, 0}; return r; }
static inline sj1 j1add(sj1 a, sj1 b) { sj1 r = {a.v + b.v, a.d + b.d, a.dd + b.dd}; return r; }
static inline sj1 j1sub(sj1 a, sj1 b) { sj1 r = {a.v - b.v, a.d - b.d, a.dd - b.dd}; return r; }
static inline sj1 j1mul(sj1 a, sj1 b) {
    sj1 r = {a.v * b.v, a.v * b.d + a.d * b.v, a.v * b.dd + 2.0 * a.d * b.d + a.dd * b.v};
    return r;
}
static inline sj1 j1div(sj1 a, sj1 b) {
    double ib = 1.0 / b.v;
    sj1 inv = {ib, -b.d * ib * ib, (2.0 * b.d * b.d * ib - b.dd) * ib * ib};
    return j1mul(a, inv);
}
static inline sj1 j1scale(sj1 a, double c) { sj1 r = {a.v * c, a.d * c, a.dd * c}; return r; }

static void ssim_window(const orc_config *cfg, double *w1) {
    int R = cfg->ssim_radius;
    double s = 0;
    for (int i = -R; i <= R; ++i) {
        w1[i + R] = exp(-(double)(i * i) / (2.0 * cfg->ssim_sigma * cfg->ssim_sigma));
        s += w1[i + R];
    }
    for (int i = 0; i < 2 * R + 1; ++i) w1[i] /= s;
}

static sj1 ssim_of(sj1 mu, double mut, sj1 ecc, double ett, sj1 ect, double C1, double C2) {
    sj1 var = j1sub(ecc, j1mul(mu, mu));
    double vart = ett - mut * mut;
    sj1 cov = j1sub(ect, j1scale(mu, mut));
    sj1 f0 = j1add(j1scale(mu, 2.0 * mut), j1c(C1));
    sj1 f1 = j1add(j1scale(cov, 2.0), j1c(C2));
    sj1 f2 = j1add(j1mul(mu, mu), j1c(mut * mut + C1));
    sj1 f3 = j1add(var, j1c(vart + C2));
    return j1div(j1mul(f0, f1), j1mul(f2, f3));
}

/* Window moments of one channel at every centre p (zero padding outside the
 * image): mom[0..4][p] = sum_q w(q - p) (x_q, y_q, x_q^2, y_q^2, x_q y_q), w the
 * separable normalised Gaussian window of ssim_window. */
static void ssim_moments(const double *X, const double *Y, int W, int H, int R, const double *w1, double *mom) {
    size_t P = (size_t)W * H;
#pragma omp parallel for schedule(static)
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            double m[5] = {0, 0, 0, 0, 0};
            for (int dy = -R; dy <= R; ++dy) {
                int qy = py + dy;
                if (qy < 0 || qy >= H) continue;
                for (int dx = -R; dx <= R; ++dx) {
                    int qx = px + dx;
                    if (qx < 0 || qx >= W) continue;
                    double w = w1[dy + R] * w1[dx + R];
                    double x = X[(size_t)qy * W + qx], y = Y[(size_t)qy * W + qx];
                    m[0] += w * x; m[1] += w * y; m[2] += w * x * x; m[3] += w * y * y; m[4] += w * x * y;
                }
            }
            for (int i = 0; i < 5; ++i) mom[i * P + (size_t)py * W + px] = m[i];
        }
}

/* Exported.  Per-pixel SSIM of every channel (the quantity L_S averages):
 * ssim [3][H][W] out; mom (may be NULL) [3][5][H][W] out, the window moments
 * (mu_x, mu_y, E x^2, E y^2, E xy) it is formed from. */
void orc_ssim_map(const double *img, const double *tgt, int W, int H, const orc_config *cfg, double *ssim,
                  double *mom_out) {
    size_t P = (size_t)W * H;
    int R = cfg->ssim_radius;
    double w1[64];
    ssim_window(cfg, w1);
    double *mom = (double *)malloc(sizeof(double) * 5 * P);
    for (int c = 0; c < 3; ++c) {
        ssim_moments(img + c * P, tgt + c * P, W, H, R, w1, mom);
        for (size_t p = 0; p < P; ++p)
            ssim[c * P + p] = ssim_of(j1c(mom[p]), mom[P + p], j1c(mom[2 * P + p]), mom[3 * P + p],
                                      j1c(mom[4 * P + p]), cfg->ssim_c1, cfg->ssim_c2).v;
        if (mom_out) memcpy(mom_out + 5 * P * c, mom, sizeof(double) * 5 * P);
    }
    free(mom);
}

/* Exported.  img, tgt: [3][H][W].  e, h: [3][H][W] out.  parts[0] = L2, parts[1] = L_S.
 * Returns L = L2 + lambda L_S. */
double orc_loss(const double *img, const double *tgt, int W, int H, const orc_config *cfg, double *e, double *h,
                double *parts) {
    size_t P = (size_t)W * H;
    double sc = 1.0 / (3.0 * (double)P);
    double L2 = 0.0, LS = 0.0;
    for (size_t i = 0; i < 3 * P; ++i) {
        double d = img[i] - tgt[i];
        L2 += 0.5 * d * d;
        if (e) e[i] = sc * d;
        if (h) h[i] = sc;
    }
    L2 *= sc;
    double lam = cfg->lambda_ssim;
    if (lam != 0.0) {
        int R = cfg->ssim_radius, WS = 2 * R + 1;
        double w1[64];
        ssim_window(cfg, w1);
        double C1 = cfg->ssim_c1, C2 = cfg->ssim_c2;
        double *mom = (double *)malloc(sizeof(double) * 5 * P);
        for (int c = 0; c < 3; ++c) {
            const double *X = img + c * P, *Y = tgt + c * P;
            ssim_moments(X, Y, W, H, R, w1, mom);
            double lsum = 0.0;
            for (size_t p = 0; p < P; ++p) {
                sj1 s = ssim_of(j1c(mom[p]), mom[P + p], j1c(mom[2 * P + p]), mom[3 * P + p], j1c(mom[4 * P + p]), C1, C2);
                lsum += 1.0 - s.v;
            }
            LS += sc * lsum;
            if (e || h) {
#pragma omp parallel for schedule(static)
                for (int qy = 0; qy < H; ++qy)
                    for (int qx = 0; qx < W; ++qx) {
                        size_t q = (size_t)qy * W + qx;
                        double x = X[q], y = Y[q];
                        double de = 0.0, dh = 0.0;
                        for (int py = qy - R; py <= qy + R; ++py) {
                            if (py < 0 || py >= H) continue;
                            for (int px = qx - R; px <= qx + R; ++px) {
                                if (px < 0 || px >= W) continue;
                                size_t p = (size_t)py * W + px;
                                double w = w1[qy - py + R] * w1[qx - px + R];
                                sj1 mu = {mom[p], w, 0.0};
                                sj1 ecc = {mom[2 * P + p], 2.0 * w * x, 2.0 * w};
                                sj1 ect = {mom[4 * P + p], w * y, 0.0};
                                sj1 s = ssim_of(mu, mom[P + p], ecc, mom[3 * P + p], ect, C1, C2);
                                de += s.d;
                                dh += s.dd;
                            }
                        }
                        (void)WS;
                        if (e) e[c * P + q] -= lam * sc * de;
                        if (h) h[c * P + q] -= lam * sc * dh;
                    }
            }
        }
        free(mom);
    }
    if (parts) {
        parts[0] = L2;
        parts[1] = LS;
    }
    return L2 + lam * LS;
}

/* ---------------------------------------------------------------------------
 * Block assembly [Eq. local_hessian_gradient]:
 *   g_y += sum_p sum_ch e_ch(p) dc_ch(p)/dy
 *   H_y += sum_p sum_ch ( h_ch(p) dc_ch/dy dc_ch/dy^T + e_ch(p) d2c_ch/dy2 )
 * With cfg->gauss_newton the second term is dropped: the Gauss-Newton block
 * sum_p sum_ch h_ch(p) dc_ch/dy dc_ch/dy^T (a local Gauss-Newton variant per
 * attribute, which the conclusion names as a cheaper position path).
 * where, for Gaussian k, c(p) = C_front + T_k (alpha_k c~_k + (1 - alpha_k) C_back_k)
 * (Eq. 3dgs regrouped around term k; T_k and C_back_k do not depend on y_k).
 * alpha_k and c~_k are evaluated as jets of y_k; the set of contributors is
 * that of the plain pass (held fixed, as derivatives of a piecewise formula).
 * Views add with weight 1 [Eq. tildel].
 *
 * Layouts (D = variable count of the group, NH = D(D+1)/2):
 *   POS/SCALE: g [3][n], H [6][n]; ROT/OPACITY: g [1][n], H [1][n];
 *   COLOR: g [3][S][n], H [3][S(S+1)/2][n] (per channel, decoupled).
 * gabs/Habs (optional) accumulate |terms| for scale-aware tolerances,
 * npix (optional) counts contributing pixels.
 * ------------------------------------------------------------------------- */
static int group_dims(int group, int S) {
    switch (group) {
    case G_POS: return 3;
    case G_ROT: return 1;
    case G_SCALE: return 3;
    case G_OPACITY: return 1;
    case G_COLOR: return S;
    }
    return 0;
}

static void accum_channelset(const orc_scene *sc, const orc_camera *cam, const orc_camera *primary,
                             const orc_config *cfg, int group, int ch, const double *e, const double *h, double *g,
                             double *Hb, double *gabs, double *Habs, int *npix) {
    int n = sc->n, S = orc_sh_count(sc->sh_degree);
    JD = group_dims(group, S);
    int D = JD, NH = jnh();
    viewset vs;
    viewset_build(&vs, sc, cam, primary, cfg, group, ch);
    int W = cam->width, H = cam->height;
    size_t P = (size_t)W * H;
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    size_t per = (size_t)n * (D + NH) * 2;
    double *tbuf = (double *)calloc((size_t)nthreads * per, sizeof(double));
    int *tcnt = (int *)calloc((size_t)nthreads * n, sizeof(int));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *tg = tbuf + tid * per;
        double *tH = tg + (size_t)n * D;
        double *tga = tH + (size_t)n * NH;
        double *tHa = tga + (size_t)n * D;
        int *tc = tcnt + (size_t)tid * n;
        contrib *list = (contrib *)malloc(sizeof(contrib) * (vs.norder + 1));
        double *cback = (double *)malloc(sizeof(double) * 3 * (vs.norder + 1));
#pragma omp for schedule(dynamic, 1)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                double C[3], T;
                int nc = pixel_pass(&vs, cfg, (double)x, (double)y, list, C, &T, NULL);
                double cb[3] = {0, 0, 0};
                for (int j = nc - 1; j >= 0; --j) {
                    const double *pl = vs.plain + list[j].k * NPJ;
                    for (int c = 0; c < 3; ++c) {
                        cback[j * 3 + c] = cb[c];
                        cb[c] = list[j].alpha * pl[6 + c] + (1.0 - list[j].alpha) * cb[c];
                    }
                }
                double ep[3], hp[3];
                for (int c = 0; c < 3; ++c) {
                    ep[c] = e[c * P + (size_t)y * W + x];
                    hp[c] = h[c * P + (size_t)y * W + x];
                }
                for (int j = 0; j < nc; ++j) {
                    int k = list[j].k;
                    const double *pj = vs.jets + (size_t)k * NPJ * vs.js;
                    jet pix0, pix1, c0, c1, c2, op, col[3];
                    junpack(&pix0, pj + 0 * vs.js);
                    junpack(&pix1, pj + 1 * vs.js);
                    junpack(&c0, pj + 2 * vs.js);
                    junpack(&c1, pj + 3 * vs.js);
                    junpack(&c2, pj + 4 * vs.js);
                    junpack(&op, pj + 5 * vs.js);
                    for (int c = 0; c < 3; ++c) junpack(&col[c], pj + (6 + c) * vs.js);
                    jet dx, dy, q, t, G, alpha;
                    jscale(&dx, &pix0, -1.0);
                    jaddc(&dx, &dx, (double)x);
                    jscale(&dy, &pix1, -1.0);
                    jaddc(&dy, &dy, (double)y);
                    jmul(&q, &dx, &dx);
                    jmul(&q, &q, &c0);
                    jmul(&t, &dx, &dy);
                    jmul(&t, &t, &c1);
                    jscale(&t, &t, 2.0);
                    jadd(&q, &q, &t);
                    jmul(&t, &dy, &dy);
                    jmul(&t, &t, &c2);
                    jadd(&q, &q, &t);
                    jscale(&q, &q, -0.5);
                    jexp(&G, &q);
                    if (list[j].clamped) jconst(&alpha, cfg->alpha_max);
                    else jmul(&alpha, &op, &G);
                    double Tk = list[j].T;
                    for (int c = 0; c < 3; ++c) {
                        /* c_ch = T_k (alpha c~ + (1 - alpha) Cb) + const */
                        jet a1, a2, cc;
                        jmul(&a1, &alpha, &col[c]);
                        jscale(&a2, &alpha, -cback[j * 3 + c]);
                        jadd(&cc, &a1, &a2);
                        jscale(&cc, &cc, Tk);
                        int kk = 0;
                        for (int a = 0; a < D; ++a) {
                            double gv = ep[c] * cc.g[a];
                            tg[(size_t)a * n + k] += gv;
                            tga[(size_t)a * n + k] += fabs(gv);
                            for (int b = a; b < D; ++b, ++kk) {
                                double t1 = hp[c] * cc.g[a] * cc.g[b];
                                double t2 = cfg->gauss_newton ? 0.0 : ep[c] * cc.h[kk];
                                tH[(size_t)kk * n + k] += t1 + t2;
                                tHa[(size_t)kk * n + k] += fabs(t1) + fabs(t2);
                            }
                        }
                    }
                    tc[k] += 1;
                }
            }
        free(list);
        free(cback);
    }
    for (int t = 0; t < nthreads; ++t) {
        double *tg = tbuf + t * per;
        double *tH = tg + (size_t)n * D;
        double *tga = tH + (size_t)n * NH;
        double *tHa = tga + (size_t)n * D;
        for (size_t i = 0; i < (size_t)n * D; ++i) {
            g[i] += tg[i];
            if (gabs) gabs[i] += tga[i];
        }
        for (size_t i = 0; i < (size_t)n * NH; ++i) {
            Hb[i] += tH[i];
            if (Habs) Habs[i] += tHa[i];
        }
        if (npix)
            for (int k = 0; k < n; ++k) npix[k] += tcnt[(size_t)t * n + k];
    }
    free(tbuf);
    free(tcnt);
    viewset_free(&vs);
}

int orc_accum(int group, const orc_scene *sc, const orc_camera *view, const orc_camera *primary,
              const orc_config *cfg, const double *e, const double *h, double *g, double *Hb, double *gabs,
              double *Habs, int *npix) {
    int save = JD;
    int n = sc->n, S = orc_sh_count(sc->sh_degree);
    if (group == G_COLOR) {
        int NH = S * (S + 1) / 2;
        for (int ch = 0; ch < 3; ++ch)
            accum_channelset(sc, view, primary, cfg, group, ch, e, h, g + (size_t)ch * S * n,
                             Hb + (size_t)ch * NH * n, gabs ? gabs + (size_t)ch * S * n : NULL,
                             Habs ? Habs + (size_t)ch * NH * n : NULL, (ch == 0) ? npix : NULL);
    } else {
        accum_channelset(sc, view, primary, cfg, group, 0, e, h, g, Hb, gabs, Habs, npix);
    }
    JD = save;
    return 0;
}

/* ---------------------------------------------------------------------------
 * Damped dense solve (H + mu m I) x = -g, m = mean |diag H|          [reading]
 * The paper fixes step size 1 with no line search and is silent on
 * indefinite blocks.  Reading: mu = mu0 * 10^i for i = 0..tries until the
 * Cholesky factorisation has only positive pivots; if none does, x = 0
 * (status 1).  A block whose gradient and Hessian are all zero (no
 * contributing pixel) gets x = 0 (status 2).
 * info[0] = mu used, info[1] = smallest |pivot| / diag over all attempts
 * made (how close the accept / reject decision was), info[2] = number of
 * failed attempts.
 * ------------------------------------------------------------------------- */
static int damped_solve(int N, const double *Hf, const double *g, const orc_config *cfg, double *x, double *info) {
    double m = 0.0, gz = 0.0;
    for (int i = 0; i < N; ++i) {
        m += fabs(Hf[i * N + i]);
        gz += fabs(g[i]);
    }
    for (int i = 0; i < N * N; ++i) gz += fabs(Hf[i]);
    for (int i = 0; i < N; ++i) x[i] = 0.0;
    if (info) { info[0] = 0; info[1] = INFINITY; info[2] = 0; }
    if (gz == 0.0) return 2;
    m /= N;
    double A[256], L[256];
    double mu = cfg->damping_mu0;
    double mg = INFINITY;
    for (int att = 0; att <= cfg->damping_tries; ++att, mu *= 10.0) {
        for (int i = 0; i < N * N; ++i) A[i] = Hf[i];
        for (int i = 0; i < N; ++i) A[i * N + i] += mu * m;
        int ok = 1;
        for (int j = 0; j < N && ok; ++j) {
            double d = A[j * N + j];
            for (int k = 0; k < j; ++k) d -= L[j * N + k] * L[j * N + k];
            double rel = fabs(d) / (fabs(A[j * N + j]) > 0 ? fabs(A[j * N + j]) : 1.0);
            if (rel < mg) mg = rel;
            if (!(d > 0.0)) { ok = 0; break; }
            L[j * N + j] = sqrt(d);
            for (int i = j + 1; i < N; ++i) {
                double s = A[i * N + j];
                for (int k = 0; k < j; ++k) s -= L[i * N + k] * L[j * N + k];
                L[i * N + j] = s / L[j * N + j];
            }
        }
        if (!ok) {
            if (info) info[2] += 1;
            continue;
        }
        double yv[16];
        for (int i = 0; i < N; ++i) {
            double s = -g[i];
            for (int k = 0; k < i; ++k) s -= L[i * N + k] * yv[k];
            yv[i] = s / L[i * N + i];
        }
        for (int i = N - 1; i >= 0; --i) {
            double s = yv[i];
            for (int k = i + 1; k < N; ++k) s -= L[k * N + i] * x[k];
            x[i] = s / L[i * N + i];
        }
        if (info) { info[0] = mu; info[1] = mg; }
        return 0;
    }
    for (int i = 0; i < N; ++i) x[i] = 0.0;
    if (info) info[1] = mg;
    return 1;
}

static void unpack_sym(int N, const double *Hp, size_t stride, double *Hf) {
    int kk = 0;
    for (int a = 0; a < N; ++a)
        for (int b = a; b < N; ++b, ++kk) {
            Hf[a * N + b] = Hp[(size_t)kk * stride];
            Hf[b * N + a] = Hp[(size_t)kk * stride];
        }
}

/* unit camera->centre direction of the primary view */
static void view_dir(const orc_camera *cam, const double p[3], double r[3]) {
    double o[3], nn = 0;
    cam_center(cam, o);
    for (int i = 0; i < 3; ++i) {
        r[i] = p[i] - o[i];
        nn += r[i] * r[i];
    }
    nn = sqrt(nn);
    for (int i = 0; i < 3; ++i) r[i] /= nn;
}

/* Position basis [Sec. 4.2 position solve]. The printed u_y is parallel to r,
 * contradicting "perpendicular to r"; reading: u_y = normalize((I - r r^T) e_y)
 * (e_x if |r_y| > 0.999), u_x = r x u_y. */
static void position_basis(const double r[3], double U[3][2]) {
    double e[3] = {0, 1, 0};
    if (fabs(r[1]) > 0.999) { e[0] = 1; e[1] = 0; }
    double d = r[0] * e[0] + r[1] * e[1] + r[2] * e[2];
    double uy[3], nn = 0;
    for (int i = 0; i < 3; ++i) {
        uy[i] = e[i] - d * r[i];
        nn += uy[i] * uy[i];
    }
    nn = sqrt(nn);
    for (int i = 0; i < 3; ++i) uy[i] /= nn;
    double ux[3] = {r[1] * uy[2] - r[2] * uy[1], r[2] * uy[0] - r[0] * uy[2], r[0] * uy[1] - r[1] * uy[0]};
    for (int i = 0; i < 3; ++i) {
        U[i][0] = ux[i];
        U[i][1] = uy[i];
    }
}

static void quat_R_plain(const double q0[4], double R[3][3]) {
    double nn = sqrt(q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2] + q0[3] * q0[3]);
    double w = q0[0] / nn, x = q0[1] / nn, y = q0[2] / nn, z = q0[3] / nn;
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
}

/* Scaling reduction [Sec. 4.2 scaling solve]. The printed relations are
 * garbled (lambda = T s drops the squares; (T^T T)^{-1} is singular).
 * Reading: lambda_i = sum_j (V M)_ij^2 s_j^2 with M = J Wr R of the PRIMARY
 * view (no low-pass) and V the eigenvectors of M diag(s^2) M^T, so
 * Tt = d lambda / d s = 2 T diag(s), T_ij = (V M)_ij^2;
 * Q = Tt^T (Tt Tt^T)^{-1} (3x2), g_l = Q^T g_s, H_l = Q^T H_s Q,
 * dl = -H_l^{-1} g_l, ds = Q dl (the Newton step restricted to row(Tt)).
 * Returns 0 ok, 3 if not in front of the primary camera or Tt is rank
 * deficient.  gap_out = min(relative eigenvalue gap, det(Tt Tt^T) /
 * (|t1|^2 |t2|^2)): how close the reduction is to degenerate (a diagnostic
 * for tolerances; it does not change the step). */
static int scale_basis(const orc_camera *cam, const orc_config *cfg, const double p[3], const double q[4],
                       const double s[3], double Q[3][2], double *gap_out) {
    const double *V = cam->viewmat;
    double t[3];
    for (int i = 0; i < 3; ++i) t[i] = V[i * 4] * p[0] + V[i * 4 + 1] * p[1] + V[i * 4 + 2] * p[2] + V[i * 4 + 3];
    double tz = depth_fp64(cam, p[0], p[1], p[2]);
    if (!(tz >= cfg->near_z)) return 3;
    double tx = t[0] / t[2], ty = t[1] / t[2], Lx = clip_lim(cam, 0), Ly = clip_lim(cam, 1);
    tx = tx > Lx ? Lx : (tx < -Lx ? -Lx : tx);
    ty = ty > Ly ? Ly : (ty < -Ly ? -Ly : ty);
    double J[2][3] = {{cam->fx / t[2], 0, -cam->fx * tx / t[2]}, {0, cam->fy / t[2], -cam->fy * ty / t[2]}};
    double R[3][3];
    quat_R_plain(q, R);
    double M[2][3];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int i = 0; i < 3; ++i) {
                double wr = 0;
                for (int j = 0; j < 3; ++j) wr += V[i * 4 + j] * R[j][b];
                acc += J[a][i] * wr;
            }
            M[a][b] = acc;
        }
    double A00 = 0, A01 = 0, A11 = 0;
    for (int j = 0; j < 3; ++j) {
        double s2 = s[j] * s[j];
        A00 += M[0][j] * M[0][j] * s2;
        A01 += M[0][j] * M[1][j] * s2;
        A11 += M[1][j] * M[1][j] * s2;
    }
    /* eigenvectors of [[A00, A01], [A01, A11]]: angle phi with tan(2 phi) = 2 A01 / (A00 - A11) */
    double tr = A00 + A11, df = A00 - A11;
    double disc = sqrt(df * df + 4 * A01 * A01);
    if (gap_out) *gap_out = (tr > 0) ? disc / tr : 0.0;
    double phi = 0.5 * atan2(2 * A01, df);
    double v0[2] = {cos(phi), sin(phi)}, v1[2] = {-sin(phi), cos(phi)};
    double Tt[2][3];
    for (int j = 0; j < 3; ++j) {
        double a = v0[0] * M[0][j] + v0[1] * M[1][j];
        double b = v1[0] * M[0][j] + v1[1] * M[1][j];
        Tt[0][j] = 2.0 * a * a * s[j];
        Tt[1][j] = 2.0 * b * b * s[j];
    }
    double G00 = 0, G01 = 0, G11 = 0;
    for (int j = 0; j < 3; ++j) {
        G00 += Tt[0][j] * Tt[0][j];
        G01 += Tt[0][j] * Tt[1][j];
        G11 += Tt[1][j] * Tt[1][j];
    }
    double det = G00 * G11 - G01 * G01;
    if (gap_out && G00 * G11 > 0 && det / (G00 * G11) < *gap_out) *gap_out = det / (G00 * G11);
    /* rank test: rows of Tt closer than ~0.06 degrees count as parallel */
    if (!(det > 1e-300) || !(det > 1e-6 * G00 * G11)) return 3;
    double I00 = G11 / det, I01 = -G01 / det, I11 = G00 / det;
    for (int j = 0; j < 3; ++j) {
        Q[j][0] = Tt[0][j] * I00 + Tt[1][j] * I01;
        Q[j][1] = Tt[0][j] * I01 + Tt[1][j] * I11;
    }
    return 0;
}

/* Exported.  The 3x2 basis B of each Gaussian's reduced solve (tests use it
 * to propagate block tolerances to steps): POS the orthonormal U
 * perpendicular to the primary view ray [Sec. 4.2 position solve], SCALE
 * Q = Tt^T (Tt Tt^T)^-1 [Sec. 4.2 scaling solve].  B_out [n][3][2] (row i,
 * column a at 6k + 2i + a); status [n]: 0 ok, 3 undefined (scaling: behind
 * the primary camera or rank-deficient Tt); gap_out [n] (may be NULL): for
 * scaling how close its reduction is to degenerate (the smaller of the
 * relative eigenvalue gap of the projected covariance and det(Tt Tt^T) /
 * (|t1|^2 |t2|^2)), infinity for position.  Returns 0, or -1 for another
 * group. */
int orc_reduced_basis(int group, const orc_scene *sc, const orc_camera *primary, const orc_config *cfg,
                      double *B_out, int *status, double *gap_out) {
    if (group != G_POS && group != G_SCALE) return -1;
    int n = sc->n;
    for (int k = 0; k < n; ++k) {
        double p[3], q[4], s[3], B[3][2] = {{0, 0}, {0, 0}, {0, 0}};
        for (int i = 0; i < 3; ++i) {
            p[i] = sc->mean[i * n + k];
            s[i] = sc->scale[i * n + k];
        }
        for (int i = 0; i < 4; ++i) q[i] = sc->quat[i * n + k];
        int st = 0;
        double gap = INFINITY;
        if (group == G_POS) {
            double r[3];
            view_dir(primary, p, r);
            position_basis(r, B);
        } else {
            st = scale_basis(primary, cfg, p, q, s, B, &gap);
        }
        if (gap_out) gap_out[k] = gap;
        for (int i = 0; i < 3; ++i)
            for (int a = 0; a < 2; ++a) B_out[6 * (size_t)k + 2 * i + a] = B[i][a];
        status[k] = st;
    }
    return 0;
}

/* Exported solve.  g/H layouts as orc_accum.  step: POS [3][n], ROT [1][n],
 * SCALE [3][n], OPACITY [1][n], COLOR [3][S][n].
 * status [n] (COLOR: [3][n]): 0 ok, 1 damping failed, 2 no contribution,
 * 3 reduction undefined.  info [3][n] (COLOR [3][3][n]) from damped_solve;
 * for SCALE info additionally holds the eigen-gap in cond slot below.
 * cond [n] (COLOR [3][n]): 2-norm condition of the damped block (fp64, from
 * the Cholesky-accepted matrix via power iterations on A and A^{-1}). */
static double cond_estimate(int N, const double *Hf, double damp) {
    /* explicit eigenvalues would need a library; use power iteration on A and
     * on A^{-1} (via Cholesky solves) — adequate for a tolerance scale. */
    double A[256], L[256], v[16], w[16];
    for (int i = 0; i < N * N; ++i) A[i] = Hf[i];
    for (int i = 0; i < N; ++i) A[i * N + i] += damp;
    for (int j = 0; j < N; ++j) {
        double d = A[j * N + j];
        for (int k = 0; k < j; ++k) d -= L[j * N + k] * L[j * N + k];
        if (!(d > 0)) return INFINITY;
        L[j * N + j] = sqrt(d);
        for (int i = j + 1; i < N; ++i) {
            double s = A[i * N + j];
            for (int k = 0; k < j; ++k) s -= L[i * N + k] * L[j * N + k];
            L[i * N + j] = s / L[j * N + j];
        }
    }
    double lmax = 0, lmin_inv = 0;
    for (int i = 0; i < N; ++i) v[i] = 1.0 + 0.1 * i;
    for (int it = 0; it < 200; ++it) {
        double nn = 0;
        for (int i = 0; i < N; ++i) {
            w[i] = 0;
            for (int j = 0; j < N; ++j) w[i] += A[i * N + j] * v[j];
            nn += w[i] * w[i];
        }
        nn = sqrt(nn);
        lmax = nn;
        for (int i = 0; i < N; ++i) v[i] = w[i] / nn;
    }
    for (int i = 0; i < N; ++i) v[i] = 1.0 - 0.05 * i;
    for (int it = 0; it < 200; ++it) {
        double y[16];
        for (int i = 0; i < N; ++i) {
            double s = v[i];
            for (int k = 0; k < i; ++k) s -= L[i * N + k] * y[k];
            y[i] = s / L[i * N + i];
        }
        for (int i = N - 1; i >= 0; --i) {
            double s = y[i];
            for (int k = i + 1; k < N; ++k) s -= L[k * N + i] * w[k];
            w[i] = s / L[i * N + i];
        }
        double nn = 0;
        for (int i = 0; i < N; ++i) nn += w[i] * w[i];
        nn = sqrt(nn);
        lmin_inv = nn;
        for (int i = 0; i < N; ++i) v[i] = w[i] / nn;
    }
    return lmax * lmin_inv;
}

/* First-order baseline on the same blocks: the step -lr g of the group's
 * gradient (g of Eq. local_hessian_gradient; opacity with the barrier's
 * gradient added), kept inside the same trust radii and bounds as the Newton
 * step: position |dp| <= trust_pos max(s) (full 3D step), rotation
 * |theta| <= trust_rot, scaling within [s / kappa, kappa s], opacity by the
 * fraction-to-boundary rule, colour per channel |dc| <= trust_color.  A
 * Gaussian with no contributing pixel (g and H zero) does not move. */
static int gradient_step(int group, const orc_scene *sc, const orc_config *cfg, const double *g, const double *Hb,
                         double *step, int *status) {
    const int n = sc->n, S = orc_sh_count(sc->sh_degree);
    const double lr = cfg->gd_lr[group];
    if (group == G_COLOR) {
        const int NH = S * (S + 1) / 2;
        for (int ch = 0; ch < 3; ++ch)
            for (int k = 0; k < n; ++k) {
                double x[16];
                for (int i = 0; i < S; ++i) x[i] = -lr * g[((size_t)ch * S + i) * n + k];
                trust_scale(S, x, cfg->trust_color);
                for (int i = 0; i < S; ++i) step[((size_t)ch * S + i) * n + k] = x[i];
                if (status) status[ch * n + k] = 0;
                (void)NH;
            }
        return 0;
    }
    const int D = group_dims(group, S), NHg = D * (D + 1) / 2;
    for (int k = 0; k < n; ++k) {
        int none = 1;
        for (int i = 0; i < D; ++i) if (g[(size_t)i * n + k] != 0.0) none = 0;
        for (int i = 0; i < NHg; ++i) if (Hb[(size_t)i * n + k] != 0.0) none = 0;
        for (int i = 0; i < D; ++i) step[(size_t)i * n + k] = 0.0;
        if (status) status[k] = none ? 2 : 0;
        if (none) continue;
        if (group == G_POS) {
            double x[3], smax = 0;
            for (int i = 0; i < 3; ++i) {
                x[i] = -lr * g[(size_t)i * n + k];
                smax = fmax(smax, sc->scale[i * n + k]);
            }
            trust_scale(3, x, cfg->trust_pos * smax);
            for (int i = 0; i < 3; ++i) step[(size_t)i * n + k] = x[i];
        } else if (group == G_ROT) {
            double x = -lr * g[k];
            trust_scale(1, &x, cfg->trust_rot);
            step[k] = x;
        } else if (group == G_SCALE) {
            for (int i = 0; i < 3; ++i) {
                const double si = sc->scale[i * n + k];
                double ns = si - lr * g[(size_t)i * n + k];
                if (ns < si / cfg->scale_trust) ns = si / cfg->scale_trust;
                if (ns > si * cfg->scale_trust) ns = si * cfg->scale_trust;
                step[(size_t)i * n + k] = ns - si;
            }
        } else { /* opacity */
            const double sg = sc->opacity[k], a = cfg->barrier_alpha, tau = cfg->frac_to_boundary;
            double ns = sg - lr * (g[k] + a * (-1.0 / sg + 1.0 / (1.0 - sg)));
            if (ns < sg - tau * sg) ns = sg - tau * sg;
            if (ns > sg + tau * (1.0 - sg)) ns = sg + tau * (1.0 - sg);
            step[k] = ns - sg;
        }
    }
    return 0;
}

int orc_solve(int group, const orc_scene *sc, const orc_camera *primary, const orc_config *cfg, const double *g,
              const double *Hb, double *step, int *status, double *info, double *cond) {
    int n = sc->n, S = orc_sh_count(sc->sh_degree);
    int nfail = 0;
    if (cfg->gd_lr[group] > 0.0) {
        if (info) memset(info, 0, sizeof(double) * 3 * (size_t)n * (group == G_COLOR ? 3 : 1));
        if (cond) memset(cond, 0, sizeof(double) * (size_t)n * (group == G_COLOR ? 3 : 1));
        return gradient_step(group, sc, cfg, g, Hb, step, status);
    }
    if (group == G_COLOR) {
        int NH = S * (S + 1) / 2;
        for (int ch = 0; ch < 3; ++ch)
            for (int k = 0; k < n; ++k) {
                double Hf[256], gv[16], x[16], inf[3];
                unpack_sym(S, Hb + ((size_t)ch * NH) * n + k, n, Hf);
                for (int i = 0; i < S; ++i) gv[i] = g[((size_t)ch * S + i) * n + k];
                int st = damped_solve(S, Hf, gv, cfg, x, inf);
                if (st == 0 && trust_scale(S, x, cfg->trust_color)) st = 1;
                for (int i = 0; i < S; ++i) step[((size_t)ch * S + i) * n + k] = x[i];
                if (status) status[ch * n + k] = st;
                if (info) for (int i = 0; i < 3; ++i) info[((size_t)ch * 3 + i) * n + k] = inf[i];
                if (cond) {
                    double m = 0;
                    for (int i = 0; i < S; ++i) m += fabs(Hf[i * S + i]);
                    m /= S;
                    cond[ch * n + k] = (st == 0) ? cond_estimate(S, Hf, inf[0] * m) : 0.0;
                }
                nfail += (st == 1);
            }
        return nfail;
    }
    for (int k = 0; k < n; ++k) {
        double p[3], q[4], s[3];
        for (int i = 0; i < 3; ++i) {
            p[i] = sc->mean[i * n + k];
            s[i] = sc->scale[i * n + k];
        }
        for (int i = 0; i < 4; ++i) q[i] = sc->quat[i * n + k];
        double inf[3] = {0, INFINITY, 0}, cnd = 0;
        int st = 0;
        if (group == G_POS) {
            double Hf[9], r[3], U[3][2], Hv[4], gv[2], dv[2];
            unpack_sym(3, Hb + k, n, Hf);
            view_dir(primary, p, r);
            position_basis(r, U);
            for (int a = 0; a < 2; ++a) {
                gv[a] = 0;
                for (int i = 0; i < 3; ++i) gv[a] += U[i][a] * g[i * n + k];
                for (int b = 0; b < 2; ++b) {
                    double acc = 0;
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j) acc += U[i][a] * Hf[i * 3 + j] * U[j][b];
                    Hv[a * 2 + b] = acc;
                }
            }
            st = damped_solve(2, Hv, gv, cfg, dv, inf);
            double smax = fmax(s[0], fmax(s[1], s[2]));
            if (st == 0 && trust_scale(2, dv, cfg->trust_pos * smax)) st = 1;
            for (int i = 0; i < 3; ++i) step[i * n + k] = U[i][0] * dv[0] + U[i][1] * dv[1];
            if (cond && st == 0) cnd = cond_estimate(2, Hv, inf[0] * 0.5 * (fabs(Hv[0]) + fabs(Hv[3])));
        } else if (group == G_ROT) {
            double Hf[1] = {Hb[k]}, gv[1] = {g[k]}, x[1];
            st = damped_solve(1, Hf, gv, cfg, x, inf);
            if (st == 0 && trust_scale(1, x, cfg->trust_rot)) st = 1;
            step[k] = x[0];
            cnd = 1.0;
        } else if (group == G_SCALE) {
            double Hf[9], Q[3][2], gap = 0;
            unpack_sym(3, Hb + k, n, Hf);
            int zero = 1;
            for (int i = 0; i < 3; ++i) if (g[i * n + k] != 0) zero = 0;
            for (int i = 0; i < 9; ++i) if (Hf[i] != 0) zero = 0;
            for (int i = 0; i < 3; ++i) step[i * n + k] = 0.0;
            if (zero) {
                st = 2;
            } else if (scale_basis(primary, cfg, p, q, s, Q, &gap) != 0) {
                st = 3;
            } else {
                double Hl[4], gl[2], dl[2];
                for (int a = 0; a < 2; ++a) {
                    gl[a] = 0;
                    for (int i = 0; i < 3; ++i) gl[a] += Q[i][a] * g[i * n + k];
                    for (int b = 0; b < 2; ++b) {
                        double acc = 0;
                        for (int i = 0; i < 3; ++i)
                            for (int j = 0; j < 3; ++j) acc += Q[i][a] * Hf[i * 3 + j] * Q[j][b];
                        Hl[a * 2 + b] = acc;
                    }
                }
                st = damped_solve(2, Hl, gl, cfg, dl, inf);
                if (st == 0 && trust_scale(2, dl, INFINITY)) st = 1;
                /* positivity of s (reading; the paper gives no rule): the update
                 * stays within [s / kappa, kappa s], kappa = scale_trust, i.e. a
                 * bounded step in log-scale (cf. the opacity fraction-to-boundary) */
                for (int i = 0; i < 3; ++i) {
                    double ds = Q[i][0] * dl[0] + Q[i][1] * dl[1];
                    double lo = s[i] / cfg->scale_trust, hi = s[i] * cfg->scale_trust;
                    double ns = s[i] + ds;
                    if (ns < lo) ns = lo;
                    if (ns > hi) ns = hi;
                    step[i * n + k] = ns - s[i];
                }
                if (cond && st == 0) cnd = cond_estimate(2, Hl, inf[0] * 0.5 * (fabs(Hl[0]) + fabs(Hl[3])));
            }
            if (cond) cond[k] = (st == 0) ? cnd : 0.0;
            if (status) status[k] = st;
            if (info) {
                info[0 * (size_t)n + k] = inf[0];
                info[1 * (size_t)n + k] = (st == 0) ? fmin(inf[1], gap) : inf[1];
                info[2 * (size_t)n + k] = inf[2];
            }
            nfail += (st == 1);
            continue;
        } else if (group == G_OPACITY) {
            /* barrier [Sec. 4.2 opacity solve]; the printed signs are
             * inconsistent; reading: B = -a (ln s + ln(1 - s)) added once per
             * group solve, B' = a(-1/s + 1/(1-s)), B'' = a(1/s^2 + 1/(1-s)^2);
             * fraction-to-boundary keeps sigma in (0,1): the new value lies in
             * [sigma - tau sigma, sigma + tau (1 - sigma)]. */
            double sg = sc->opacity[k];
            double gv[1] = {g[k]}, Hf[1] = {Hb[k]}, x[1] = {0};
            if (gv[0] == 0.0 && Hf[0] == 0.0) {
                st = 2;
                inf[1] = INFINITY;
            } else {
                double a = cfg->barrier_alpha;
                gv[0] += a * (-1.0 / sg + 1.0 / (1.0 - sg));
                Hf[0] += a * (1.0 / (sg * sg) + 1.0 / ((1.0 - sg) * (1.0 - sg)));
                st = damped_solve(1, Hf, gv, cfg, x, inf);
                if (st == 0 && trust_scale(1, x, INFINITY)) st = 1;
            }
            double tau = cfg->frac_to_boundary;
            double lo = sg - tau * sg, hi = sg + tau * (1.0 - sg);
            double ns = sg + x[0];
            if (ns < lo) ns = lo;
            if (ns > hi) ns = hi;
            step[k] = (st == 0) ? ns - sg : 0.0;
            cnd = 1.0;
        }
        if (status) status[k] = st;
        if (info) for (int i = 0; i < 3; ++i) info[(size_t)i * n + k] = inf[i];
        if (cond) cond[k] = (st == 0) ? cnd : 0.0;
        nfail += (st == 1);
    }
    return nfail;
}

/* Exported apply [Sec. 4.2: linear updates; q <- dq q for rotation]. */
void orc_apply(int group, orc_scene *sc, const orc_camera *primary, const orc_config *cfg, const double *step) {
    int n = sc->n, S = orc_sh_count(sc->sh_degree);
    for (int k = 0; k < n; ++k) {
        if (group == G_POS) {
            for (int i = 0; i < 3; ++i) sc->mean[i * n + k] += step[i * n + k];
        } else if (group == G_ROT) {
            double p[3], a[3], q0[4];
            for (int i = 0; i < 3; ++i) p[i] = sc->mean[i * n + k];
            for (int i = 0; i < 4; ++i) q0[i] = sc->quat[i * n + k];
            view_dir(primary, p, a);
            double th = step[k], cw = cos(0.5 * th), sw = sin(0.5 * th);
            double adotv = a[0] * q0[1] + a[1] * q0[2] + a[2] * q0[3];
            double axv[3] = {a[1] * q0[3] - a[2] * q0[2], a[2] * q0[1] - a[0] * q0[3], a[0] * q0[2] - a[1] * q0[1]};
            double qn[4];
            qn[0] = cw * q0[0] - sw * adotv;
            for (int i = 0; i < 3; ++i) qn[1 + i] = cw * q0[1 + i] + sw * (q0[0] * a[i] + axv[i]);
            double nn = sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
            for (int i = 0; i < 4; ++i) sc->quat[i * n + k] = qn[i] / nn;
        } else if (group == G_SCALE) {
            for (int i = 0; i < 3; ++i) {
                double v = sc->scale[i * n + k] + step[i * n + k];
                sc->scale[i * n + k] = v > cfg->scale_min ? v : cfg->scale_min;
            }
        } else if (group == G_OPACITY) {
            sc->opacity[k] += step[k];
        } else if (group == G_COLOR) {
            for (int i = 0; i < 3 * S; ++i) sc->sh[(size_t)i * n + k] += step[(size_t)i * n + k];
        }
    }
}

/* ---------------------------------------------------------------------------
 * Data preparation [Sec. 4.1]: bounding sphere of the means (reading: centre
 * = centre of their axis-aligned box, radius = largest distance to a mean),
 * camera centres projected radially onto it, distance = great-circle angle,
 * K nearest by (angle, camera index).
 * ------------------------------------------------------------------------- */
void orc_bounding_sphere(const orc_scene *sc, double out[4]) {
    int n = sc->n;
    double lo[3], hi[3];
    for (int i = 0; i < 3; ++i) { lo[i] = INFINITY; hi[i] = -INFINITY; }
    for (int k = 0; k < n; ++k)
        for (int i = 0; i < 3; ++i) {
            double v = sc->mean[i * n + k];
            if (v < lo[i]) lo[i] = v;
            if (v > hi[i]) hi[i] = v;
        }
    for (int i = 0; i < 3; ++i) out[i] = 0.5 * (lo[i] + hi[i]);
    double r2 = 0;
    for (int k = 0; k < n; ++k) {
        double d = 0;
        for (int i = 0; i < 3; ++i) {
            double t = sc->mean[i * n + k] - out[i];
            d += t * t;
        }
        if (d > r2) r2 = d;
    }
    out[3] = sqrt(r2);
}

static const double *g_knn_dist;
static int cmp_knn(const void *a, const void *b) {
    int i = *(const int *)a, j = *(const int *)b;
    if (g_knn_dist[i] < g_knn_dist[j]) return -1;
    if (g_knn_dist[i] > g_knn_dist[j]) return 1;
    return (i < j) ? -1 : (i > j);
}

/* centres [ncam][3]; out [ncam][K]; dist_out optional [ncam][ncam] */
int orc_knn(int ncam, const double *centres, const double sphere[4], int K, int *out, double *dist_out) {
    double *u = (double *)malloc(sizeof(double) * 3 * ncam);
    for (int i = 0; i < ncam; ++i) {
        double nn = 0;
        for (int a = 0; a < 3; ++a) {
            u[i * 3 + a] = centres[i * 3 + a] - sphere[a];
            nn += u[i * 3 + a] * u[i * 3 + a];
        }
        nn = sqrt(nn);
        for (int a = 0; a < 3; ++a) u[i * 3 + a] /= nn;
    }
    double *dist = (double *)malloc(sizeof(double) * ncam);
    int *idx = (int *)malloc(sizeof(int) * ncam);
    for (int i = 0; i < ncam; ++i) {
        int m = 0;
        for (int j = 0; j < ncam; ++j) {
            double c = u[i * 3] * u[j * 3] + u[i * 3 + 1] * u[j * 3 + 1] + u[i * 3 + 2] * u[j * 3 + 2];
            if (c > 1) c = 1;
            if (c < -1) c = -1;
            dist[j] = sphere[3] * acos(c);
            if (dist_out) dist_out[(size_t)i * ncam + j] = dist[j];
            if (j != i) idx[m++] = j;
        }
        g_knn_dist = dist;
        qsort(idx, m, sizeof(int), cmp_knn);
        for (int k = 0; k < K; ++k) out[i * K + k] = (k < m) ? idx[k] : -1;
    }
    free(u);
    free(dist);
    free(idx);
    return 0;
}

/* Secondary targets are downsampled [Sec. 4.3]; reading: integer factor f,
 * f x f box filter, intrinsics scaled so pixel centres stay consistent. */
void orc_downsample_camera(const orc_camera *in, int f, orc_camera *out) {
    *out = *in;
    out->width = in->width / f;
    out->height = in->height / f;
    out->fx = in->fx / f;
    out->fy = in->fy / f;
    out->cx = (in->cx + 0.5) / f - 0.5;
    out->cy = (in->cy + 0.5) / f - 0.5;
}

void orc_downsample_image(const double *in, int W, int H, int f, double *out) {
    int W2 = W / f, H2 = H / f;
    for (int c = 0; c < 3; ++c)
        for (int y = 0; y < H2; ++y)
            for (int x = 0; x < W2; ++x) {
                double s = 0;
                for (int dy = 0; dy < f; ++dy)
                    for (int dx = 0; dx < f; ++dx) s += in[(size_t)c * W * H + (size_t)(y * f + dy) * W + x * f + dx];
                out[(size_t)c * W2 * H2 + (size_t)y * W2 + x] = s / (f * f);
            }
}

/* ---------------------------------------------------------------------------
 * One sweep for primary image t [Sec. 4.2 group order, Sec. 4.3 Eq. tildel]:
 * for each group in cfg->group_order (the paper's order by default: position,
 * rotation, scaling, opacity, colour):
 * render the primary (full resolution) and its K secondaries (downsampled),
 * accumulate the group's blocks over these views, solve, apply.
 * targets: ncam images [3][H][W] at full resolution (all cameras same size).
 * knn [ncam][K].  losses_out [5] = primary loss before each group's update
 * (indexed by group, not by position in the order).
 * ------------------------------------------------------------------------- */
int orc_sweep(orc_scene *sc, const orc_camera *cams, const double *targets, int ncam, const int *knn, int t,
              const orc_config *cfg, double *losses_out, int *nfail_out) {
    int n = sc->n, S = orc_sh_count(sc->sh_degree);
    int K = cfg->knn_k, f = cfg->downsample;
    int W = cams[t].width, H = cams[t].height;
    size_t P = (size_t)W * H;
    double *img = (double *)malloc(sizeof(double) * 3 * P);
    double *tg = (double *)malloc(sizeof(double) * 3 * P);
    double *e = (double *)malloc(sizeof(double) * 3 * P);
    double *h = (double *)malloc(sizeof(double) * 3 * P);
    size_t gmax = (size_t)3 * S * n, hmax = (size_t)3 * (S * (S + 1) / 2) * n;
    if (hmax < (size_t)6 * n) hmax = (size_t)6 * n;
    double *g = (double *)malloc(sizeof(double) * gmax);
    double *Hb = (double *)malloc(sizeof(double) * hmax);
    double *step = (double *)malloc(sizeof(double) * gmax);
    int nfail = 0;
    if (cfg->group_jacobi) {
        /* Jacobi over groups (the single-render variant): every view rendered
         * once, each group's g and H accumulated from that render, all groups
         * solved at the start state, then applied: the other groups first and
         * the position last (the rotation step turns about the primary's view
         * direction through the centre before it moves).  losses_out: the
         * primary loss in the slot of the first group of the order. */
        double *gj[5], *Hj[5], *sj[5];
        for (int q = 0; q < 5; ++q) {
            gj[q] = (double *)calloc(gmax, sizeof(double));
            Hj[q] = (double *)calloc(hmax, sizeof(double));
            sj[q] = (double *)calloc(gmax, sizeof(double));
        }
        if (losses_out) for (int q = 0; q < 5; ++q) losses_out[q] = 0.0;
        for (int vi = 0; vi <= K; ++vi) {
            int v = (vi == 0) ? t : knn[t * K + (vi - 1)];
            if (v < 0) continue;
            orc_camera cv = cams[v];
            const double *tgt = targets + (size_t)v * 3 * P;
            int Wv = W, Hv = H;
            if (vi > 0 && f > 1) {
                orc_downsample_camera(&cams[v], f, &cv);
                orc_downsample_image(tgt, W, H, f, tg);
                tgt = tg;
                Wv = cv.width;
                Hv = cv.height;
            }
            orc_render(sc, &cv, cfg, img, NULL, NULL, NULL);
            double L = orc_loss(img, tgt, Wv, Hv, cfg, e, h, NULL);
            if (vi == 0 && losses_out) losses_out[cfg->group_order[0]] = L;
            for (int q = 0; q < 5; ++q) orc_accum(q, sc, &cv, &cams[t], cfg, e, h, gj[q], Hj[q], NULL, NULL, NULL);
        }
        for (int gi = 0; gi < 5; ++gi) {
            const int q = cfg->group_order[gi];
            nfail += orc_solve(q, sc, &cams[t], cfg, gj[q], Hj[q], sj[q], NULL, NULL, NULL);
        }
        for (int gi = 0; gi < 5; ++gi) {
            const int q = cfg->group_order[gi];
            if (q != G_POS) orc_apply(q, sc, &cams[t], cfg, sj[q]);
        }
        orc_apply(G_POS, sc, &cams[t], cfg, sj[G_POS]);
        for (int q = 0; q < 5; ++q) {
            free(gj[q]);
            free(Hj[q]);
            free(sj[q]);
        }
        if (nfail_out) *nfail_out = nfail;
        free(img); free(tg); free(e); free(h); free(g); free(Hb); free(step);
        return 0;
    }
    for (int gi = 0; gi < 5; ++gi) {
        const int group = cfg->group_order[gi];
        memset(g, 0, sizeof(double) * gmax);
        memset(Hb, 0, sizeof(double) * hmax);
        for (int vi = 0; vi <= K; ++vi) {
            int v = (vi == 0) ? t : knn[t * K + (vi - 1)];
            if (v < 0) continue;
            orc_camera cv = cams[v];
            const double *tgt = targets + (size_t)v * 3 * P;
            int Wv = W, Hv = H;
            if (vi > 0 && f > 1) {
                orc_downsample_camera(&cams[v], f, &cv);
                orc_downsample_image(tgt, W, H, f, tg);
                tgt = tg;
                Wv = cv.width;
                Hv = cv.height;
            }
            orc_render(sc, &cv, cfg, img, NULL, NULL, NULL);
            double L = orc_loss(img, tgt, Wv, Hv, cfg, e, h, NULL);
            if (vi == 0 && losses_out) losses_out[group] = L;
            orc_accum(group, sc, &cv, &cams[t], cfg, e, h, g, Hb, NULL, NULL, NULL);
        }
        nfail += orc_solve(group, sc, &cams[t], cfg, g, Hb, step, NULL, NULL, NULL);
        orc_apply(group, sc, &cams[t], cfg, step);
    }
    if (nfail_out) *nfail_out = nfail;
    free(img); free(tg); free(e); free(h); free(g); free(Hb); free(step);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Tile coverage for the binning pin.  touch [ntiles][n]: 1 if some pixel of
 * the tile composites the Gaussian (the FP32 decision q <= l), else 0.
 * rect [4][n]: the
 * support box in pixels from the reading "support = { sigma G >= alpha_min }"
 * (half extents sqrt(2 ln(sigma / alpha_min) Sigma_ii)) as x0 y0 x1 y1.
 * ------------------------------------------------------------------------- */
int orc_tile_touch(const orc_scene *sc, const orc_camera *cam, const orc_config *cfg, int tile, unsigned char *touch,
                   double *rect) {
    int save = JD;
    JD = 0;
    viewset vs;
    viewset_build(&vs, sc, cam, cam, cfg, G_VALUES, 0);
    int W = cam->width, H = cam->height, n = sc->n;
    int tx = (W + tile - 1) / tile, ty = (H + tile - 1) / tile;
    memset(touch, 0, (size_t)tx * ty * n);
    for (int oi = 0; oi < vs.norder; ++oi) {
        int k = vs.order[oi];
        const double *pl = vs.plain + k * NPJ;
        double l = 2.0 * log(pl[5] / cfg->alpha_min);
        double rx = sqrt(l * vs.sig[k * 3 + 0]), ry = sqrt(l * vs.sig[k * 3 + 2]);
        if (rect) {
            rect[0 * n + k] = pl[0] - rx;
            rect[1 * n + k] = pl[1] - ry;
            rect[2 * n + k] = pl[0] + rx;
            rect[3 * n + k] = pl[1] + ry;
        }
    }
    /* one thread per tile, so every touch entry has a single writer */
#pragma omp parallel for schedule(dynamic, 1)
    for (int tid = 0; tid < tx * ty; ++tid) {
        int x0 = (tid % tx) * tile, y0 = (tid / tx) * tile;
        for (int y = y0; y < y0 + tile && y < H; ++y)
            for (int x = x0; x < x0 + tile && x < W; ++x)
                for (int oi = 0; oi < vs.norder; ++oi) {
                    int k = vs.order[oi];
                    const dec32 *D = vs.dec + k;
                    float q32 = d_quad(D->ca, D->cb, D->cc, (float)x - D->px, (float)y - D->py);
                    if (q32 <= D->l) touch[(size_t)tid * n + k] = 1;
                }
    }
    viewset_free(&vs);
    JD = save;
    return 0;
}

/* Exported.  The FP32 decision records of a view, out [18][n] in the row
 * layout of the library's projection dump: pix_x pix_y ca cb cc sigma, three
 * zero rows (colour is not a decision), depth key, touched, l, lmax, k2, ry,
 * the two tile-rectangle words (bit patterns) and 0; Gaussians that are culled
 * or below alpha_min have all-zero rows except the depth key. */
int orc_dec32(const orc_scene *sc, const orc_camera *cam, const orc_config *cfg, float *out) {
    int save = JD;
    JD = 0;
    viewset vs;
    viewset_build(&vs, sc, cam, cam, cfg, G_VALUES, 0);
    int n = sc->n;
    memset(out, 0, sizeof(float) * 18 * (size_t)n);
    for (int k = 0; k < n; ++k) out[9 * (size_t)n + k] = vs.key[k];
    for (int i = 0; i < vs.norder; ++i) {
        int k = vs.order[i];
        const dec32 *D = vs.dec + k;
        unsigned lo = D->rect_lo, hi = D->rect_hi;
        float rl, rh;
        memcpy(&rl, &lo, 4);
        memcpy(&rh, &hi, 4);
        float v[18] = {D->px, D->py, D->ca, D->cb, D->cc, (float)sc->opacity[k], 0, 0, 0, vs.key[k],
                       (float)D->touched, D->l, D->lmax, D->k2, D->ry, rl, rh, 0};
        for (int r = 0; r < 18; ++r) out[(size_t)r * n + k] = v[r];
    }
    viewset_free(&vs);
    JD = save;
    return 0;
}

/* Exported.  Tile binning and per-tile depth order [Sec. 3], by plain loops:
 * for every Gaussian in the global (key, index) order and every 16x16 tile of
 * its support box, the tile lists the Gaussian when the FP32 support test
 * reaches one of the tile's pixels.  ranges [ntiles][2] = [start, end) into
 * ids (capacity cap).  Returns the number of listed pairs (may exceed cap:
 * then only the first cap are written). */
long long orc_tile_lists(const orc_scene *sc, const orc_camera *cam, const orc_config *cfg, unsigned *ranges,
                         unsigned *ids, long long cap) {
    int save = JD;
    JD = 0;
    viewset vs;
    viewset_build(&vs, sc, cam, cam, cfg, G_VALUES, 0);
    const int T = 16, tx = (cam->width + T - 1) / T, ty = (cam->height + T - 1) / T, nt = tx * ty;
    long long *cnt = (long long *)calloc((size_t)nt + 1, sizeof(long long));
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) { /* exclusive prefix sums -> starts */
            long long acc = 0;
            for (int t = 0; t < nt; ++t) {
                long long c = cnt[t];
                ranges[2 * t] = (unsigned)acc;
                ranges[2 * t + 1] = (unsigned)(acc + c);
                cnt[t] = acc;
                acc += c;
            }
            cnt[nt] = acc;
        }
        for (int i = 0; i < vs.norder; ++i) {
            int k = vs.order[i];
            const dec32 *D = vs.dec + k;
            if (D->touched == 0u) continue;
            unsigned x0 = D->rect_lo & 0xFFFFu, y0 = D->rect_lo >> 16, x1 = D->rect_hi & 0xFFFFu, y1 = D->rect_hi >> 16;
            for (unsigned yy = y0; yy < y1; ++yy)
                for (unsigned xx = x0; xx < x1; ++xx) {
                    if (!d_support_reaches(D, (float)(xx * T), (float)(yy * T), (float)T)) continue;
                    int t = (int)(yy * (unsigned)tx + xx);
                    if (pass == 0) cnt[t]++;
                    else {
                        if (cnt[t] < cap) ids[cnt[t]] = (unsigned)k;
                        cnt[t]++;
                    }
                }
        }
    }
    long long total = 0;
    for (int t = 0; t < nt; ++t) total += ranges[2 * t + 1] - ranges[2 * t];
    free(cnt);
    viewset_free(&vs);
    JD = save;
    return total;
}

/* exported for tests: the sorted global order of a view */
int orc_order(const orc_scene *sc, const orc_camera *cam, const orc_config *cfg, int *order_out) {
    int save = JD;
    JD = 0;
    viewset vs;
    viewset_build(&vs, sc, cam, cam, cfg, G_VALUES, 0);
    for (int i = 0; i < vs.norder; ++i) order_out[i] = vs.order[i];
    int m = vs.norder;
    viewset_free(&vs);
    JD = save;
    return m;
}
