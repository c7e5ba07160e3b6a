/*
 * lr_oracle_quad.c -- the FP64 oracle (lr_oracle.c) compiled with every `double` widened to IEEE
 * binary128 (_Float128, 113-bit significand), for one purpose: measuring how far the FP64 oracle
 * itself is from the exact result of the same algorithm on the same FP64 inputs.
 *
 * TEST INFRASTRUCTURE ONLY (like lr_oracle.c): only the tests load it.
 *
 * Nothing here restates the method: the oracle's own source is included with `double` and the
 * libm calls it makes (sqrt, floor, ceil, fabs, sin, cos) mapped to their binary128 versions, so
 * the steps, their order and every constant are those of lr_oracle.c.  The functions below only
 * convert the FP64 inputs to binary128 (exactly), run the oracle's projection, TDI and adjoint
 * steps, and round the results to FP64 once.  Their rounding error is then ~2^-113 relative per
 * operation instead of 2^-53, so |oracle64 - oracle128| is the FP64 oracle's own rounding error
 * to within 2^-60 of it.
 */
#define __STDC_WANT_IEC_60559_TYPES_EXT__ 1
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define double _Float128
#define sqrt sqrtf128
#define floor floorf128
#define ceil ceilf128
#define fabs fabsf128
#define sin sinf128
#define cos cosf128
#define atan atanf128
#include "lr_oracle.c"
#undef double
#undef sqrt
#undef floor
#undef ceil
#undef fabs
#undef sin
#undef cos
#undef atan

#define ORQ_API __attribute__((visibility("default")))

typedef _Float128 q_t;

static q_t *orq_widen(const double *a, int64_t n)
{
    q_t *q = (q_t *)malloc(sizeof(q_t) * (size_t)(n > 0 ? n : 1));
    if (q)
        for (int64_t i = 0; i < n; ++i) q[i] = (q_t)a[i];
    return q;
}

static void orq_narrow(const q_t *q, int64_t n, double *a)
{
    for (int64_t i = 0; i < n; ++i) a[i] = (double)q[i];
}

/* binary128 orbit from FP64 knots, positions [9][nk] and delays [6][nk] (NULL: light-time solve) */
static void *orq_orbit(const double *tk, int64_t nk, const double *pos, const double *delays, int bc)
{
    q_t *qt = orq_widen(tk, nk), *qp = orq_widen(pos, 9 * nk), *qd = delays ? orq_widen(delays, 6 * nk) : NULL;
    void *o = NULL;
    int st = 0;
    if (qt && qp && (qd || !delays)) o = orc_orbit_new(qt, nk, qp, qd, bc, &st);
    free(qt);
    free(qp);
    free(qd);
    return o;
}

ORQ_API int orq_set_threads(int n) { return orc_set_threads(n); }

/* X, Y, Z [3][N] of the fused response (projection orbit = TDI orbit), rounded once to FP64 */
ORQ_API int orq_response(int p, int gen, int delay_mode, double dt, double t0, int64_t N,
                         const double *tk, int64_t nk, const double *pos, const double *delays, int bc,
                         const double *hp, const double *hc, int64_t nh, double t0h,
                         double lam, double beta, double psi, double *xyz)
{
    void *o = orq_orbit(tk, nk, pos, delays, bc);
    q_t *qhp = orq_widen(hp, nh), *qhc = orq_widen(hc, nh);
    q_t *y = (q_t *)malloc(sizeof(q_t) * (size_t)(6 * N)), *x = (q_t *)malloc(sizeof(q_t) * (size_t)(3 * N));
    int st = -2;
    if (o && qhp && qhc && y && x) {
        st = orc_project(p, (q_t)dt, (q_t)t0, N, o, qhp, qhc, nh, (q_t)t0h, (q_t)lam, (q_t)beta, (q_t)psi, y);
        if (!st) st = orc_tdi(p, gen, delay_mode, (q_t)dt, (q_t)t0, N, o, y, x);
        if (!st) orq_narrow(x, 3 * N, xyz);
    }
    orc_orbit_free(o);
    free(qhp);
    free(qhc);
    free(y);
    free(x);
    return st;
}

/* gradient of <g_xyz, R(h)> with respect to h+, hx ([nh] each) and (lambda, beta, psi) */
ORQ_API int orq_backward(int p, int gen, int delay_mode, double dt, double t0, int64_t N,
                         const double *tk, int64_t nk, const double *pos, const double *delays, int bc,
                         const double *hp, const double *hc, int64_t nh, double t0h,
                         double lam, double beta, double psi, const double *gxyz,
                         double *ghp, double *ghc, double *gsky)
{
    void *o = orq_orbit(tk, nk, pos, delays, bc);
    q_t *qhp = orq_widen(hp, nh), *qhc = orq_widen(hc, nh), *qg = orq_widen(gxyz, 3 * N);
    q_t *gy = (q_t *)malloc(sizeof(q_t) * (size_t)(6 * N));
    q_t *a = (q_t *)malloc(sizeof(q_t) * (size_t)nh), *b = (q_t *)malloc(sizeof(q_t) * (size_t)nh);
    q_t g3[3];
    int st = -2;
    if (o && qhp && qhc && qg && gy && a && b) {
        st = orc_tdi_adjoint(p, gen, delay_mode, (q_t)dt, (q_t)t0, N, o, qg, gy);
        if (!st) st = orc_project_adjoint(p, (q_t)dt, (q_t)t0, N, o, nh, (q_t)t0h, (q_t)lam, (q_t)beta, (q_t)psi,
                                          gy, a, b);
        if (!st) st = orc_sky_gradient(p, (q_t)dt, (q_t)t0, N, o, qhp, qhc, nh, (q_t)t0h, (q_t)lam, (q_t)beta,
                                       (q_t)psi, gy, g3);
        if (!st) {
            orq_narrow(a, nh, ghp);
            orq_narrow(b, nh, ghc);
            orq_narrow(g3, 3, gsky);
        }
    }
    orc_orbit_free(o);
    free(qhp);
    free(qhc);
    free(qg);
    free(gy);
    free(a);
    free(b);
    return st;
}

/* X, Y, Z [3][nidx] at selected output indices (the oracle's windowed evaluator), for sampled
 * checks of long series */
ORQ_API int orq_response_at(int p, int gen, int delay_mode, double dt, double t0, int64_t N,
                            const double *tk, int64_t nk, const double *pos, const double *delays, int bc,
                            const double *hp, const double *hc, int64_t nh, double t0h,
                            double lam, double beta, double psi, const int64_t *idx, int64_t nidx, double *xyz)
{
    void *o = orq_orbit(tk, nk, pos, delays, bc);
    q_t *qhp = orq_widen(hp, nh), *qhc = orq_widen(hc, nh);
    q_t *x = (q_t *)malloc(sizeof(q_t) * (size_t)(3 * nidx > 0 ? 3 * nidx : 1));
    int st = -2;
    if (o && qhp && qhc && x) {
        st = orc_response_at(p, gen, delay_mode, (q_t)dt, (q_t)t0, N, o, o, qhp, qhc, nh, (q_t)t0h, (q_t)lam,
                             (q_t)beta, (q_t)psi, idx, nidx, x, 0);
        if (!st) orq_narrow(x, 3 * nidx, xyz);
    }
    orc_orbit_free(o);
    free(qhp);
    free(qhc);
    free(x);
    return st;
}

/* Galactic binary polarisations [n] at t0 + j dt (the oracle's formula in binary128, rounded once) */
ORQ_API void orq_gb_polarisations(double A, double f0, double fdot, double fddot, double phi0, double iota,
                                  double t0, double dt, int64_t n, double *hp, double *hc)
{
    q_t *a = (q_t *)malloc(sizeof(q_t) * (size_t)(n > 0 ? n : 1)), *b = (q_t *)malloc(sizeof(q_t) * (size_t)(n > 0 ? n : 1));
    if (!a || !b) {
        free(a);
        free(b);
        return;
    }
    orc_gb_polarisations((q_t)A, (q_t)f0, (q_t)fdot, (q_t)fddot, (q_t)phi0, (q_t)iota, (q_t)t0, (q_t)dt, n, a, b);
    orq_narrow(a, n, hp);
    orq_narrow(b, n, hc);
    free(a);
    free(b);
}
