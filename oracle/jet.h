/*
 * Second-order forward-mode "jets" (value, gradient, packed Hessian) in FP64.
 *
 * TEST INFRASTRUCTURE ONLY: part of the CPU oracle. Nothing in the product
 * path includes this file.
 *
 * A jet carries f, df/dy_i and d2f/dy_i dy_j (i <= j, packed row-major upper
 * triangle) for up to JMAX free variables y.  Every arithmetic rule below is
 * the ordinary product / quotient / chain rule truncated at second order, so
 * a function written once with jets yields the exact first and second
 * derivatives that the local Newton blocks (Eq. local_hessian_gradient) need,
 * without any hand-derived derivative table.
 *
 * The number of active variables JD is a global set by the caller before a
 * (possibly OpenMP-parallel) region and left unchanged inside it.
 */
#ifndef GS2_ORACLE_JET_H
#define GS2_ORACLE_JET_H

#include <math.h>
#include <string.h>

#define JMAX 16
#define JHMAX (JMAX * (JMAX + 1) / 2)

typedef struct {
    double v;
    double g[JMAX];
    double h[JHMAX];
} jet;

extern int JD; /* active variable count, 0..JMAX */

static inline int jnh(void) { return JD * (JD + 1) / 2; }

static inline void jconst(jet *r, double c) {
    r->v = c;
    for (int i = 0; i < JD; ++i) r->g[i] = 0.0;
    for (int i = 0, nh = jnh(); i < nh; ++i) r->h[i] = 0.0;
}

static inline void jvar(jet *r, double value, int i) {
    jconst(r, value);
    r->g[i] = 1.0;
}

static inline void jcopy(jet *r, const jet *a) {
    r->v = a->v;
    for (int i = 0; i < JD; ++i) r->g[i] = a->g[i];
    for (int i = 0, nh = jnh(); i < nh; ++i) r->h[i] = a->h[i];
}

/* r = a + b */
static inline void jadd(jet *r, const jet *a, const jet *b) {
    r->v = a->v + b->v;
    for (int i = 0; i < JD; ++i) r->g[i] = a->g[i] + b->g[i];
    for (int i = 0, nh = jnh(); i < nh; ++i) r->h[i] = a->h[i] + b->h[i];
}

/* r = a - b */
static inline void jsub(jet *r, const jet *a, const jet *b) {
    r->v = a->v - b->v;
    for (int i = 0; i < JD; ++i) r->g[i] = a->g[i] - b->g[i];
    for (int i = 0, nh = jnh(); i < nh; ++i) r->h[i] = a->h[i] - b->h[i];
}

/* r = c * a (c a plain constant) */
static inline void jscale(jet *r, const jet *a, double c) {
    r->v = c * a->v;
    for (int i = 0; i < JD; ++i) r->g[i] = c * a->g[i];
    for (int i = 0, nh = jnh(); i < nh; ++i) r->h[i] = c * a->h[i];
}

/* r = a + c (c a plain constant) */
static inline void jaddc(jet *r, const jet *a, double c) {
    jcopy(r, a);
    r->v += c;
}

/* r += c * a */
static inline void jaxpy(jet *r, double c, const jet *a) {
    r->v += c * a->v;
    for (int i = 0; i < JD; ++i) r->g[i] += c * a->g[i];
    for (int i = 0, nh = jnh(); i < nh; ++i) r->h[i] += c * a->h[i];
}

/* r = a * b (product rule to second order); r may alias a or b */
static inline void jmul(jet *r, const jet *a, const jet *b) {
    jet t;
    t.v = a->v * b->v;
    for (int i = 0; i < JD; ++i) t.g[i] = a->v * b->g[i] + b->v * a->g[i];
    int k = 0;
    for (int i = 0; i < JD; ++i)
        for (int j = i; j < JD; ++j, ++k)
            t.h[k] = a->v * b->h[k] + b->v * a->h[k] + a->g[i] * b->g[j] + a->g[j] * b->g[i];
    jcopy(r, &t);
}

/* r = f(a) given f(a.v), f'(a.v), f''(a.v) (chain rule to second order) */
static inline void jchain(jet *r, const jet *a, double f0, double f1, double f2) {
    jet t;
    t.v = f0;
    for (int i = 0; i < JD; ++i) t.g[i] = f1 * a->g[i];
    int k = 0;
    for (int i = 0; i < JD; ++i)
        for (int j = i; j < JD; ++j, ++k)
            t.h[k] = f1 * a->h[k] + f2 * a->g[i] * a->g[j];
    jcopy(r, &t);
}

static inline void jrecip(jet *r, const jet *a) {
    double x = a->v;
    jchain(r, a, 1.0 / x, -1.0 / (x * x), 2.0 / (x * x * x));
}

/* r = a / b */
static inline void jdiv(jet *r, const jet *a, const jet *b) {
    jet ib;
    jrecip(&ib, b);
    jmul(r, a, &ib);
}

static inline void jexp(jet *r, const jet *a) {
    double e = exp(a->v);
    jchain(r, a, e, e, e);
}

static inline void jsqrt(jet *r, const jet *a) {
    double s = sqrt(a->v);
    jchain(r, a, s, 0.5 / s, -0.25 / (s * a->v));
}

static inline void jsin(jet *r, const jet *a) {
    jchain(r, a, sin(a->v), cos(a->v), -sin(a->v));
}

static inline void jcos(jet *r, const jet *a) {
    jchain(r, a, cos(a->v), -sin(a->v), -cos(a->v));
}

/* dynamic packing: a jet over JD variables occupies jsize() doubles */
static inline int jsize(void) { return 1 + JD + jnh(); }

static inline void jpack(double *dst, const jet *a) {
    dst[0] = a->v;
    for (int i = 0; i < JD; ++i) dst[1 + i] = a->g[i];
    for (int i = 0, nh = jnh(); i < nh; ++i) dst[1 + JD + i] = a->h[i];
}

static inline void junpack(jet *a, const double *src) {
    a->v = src[0];
    for (int i = 0; i < JD; ++i) a->g[i] = src[1 + i];
    for (int i = 0, nh = jnh(); i < nh; ++i) a->h[i] = src[1 + JD + i];
}

#endif
