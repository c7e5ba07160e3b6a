/*
 * lr_oracle.c -- plain, slow, FP64 CPU oracle of the generic LISA time-domain response
 * (Katz, Bayle, Chua & Vallisneri, "Assessing the data-analysis impact of LISA orbit
 * approximations using a GPU-accelerated response model", arXiv:2204.06633).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file; only the
 * tests, the smoke check and the benchmark's CPU-baseline arm load it.  It shares no
 * code, table or constant generator with the CUDA library.
 *
 * Every function follows the paper's definitions step by step, in FP64, with no blocking,
 * fusion or reordering:
 *   - sky basis and wave frame ............. Sec. "Reference frames" (e_r, e_theta, e_phi;
 *                                            k = -e_r, u = -e_phi, v = -e_theta)
 *   - antenna patterns ...................... Eq. (projected-strain-ssb) and the xi+, xix
 *                                            definitions that follow it
 *   - polarisation angle psi ............... the rotation by 2 psi of Sec. "Template
 *                                            generation", applied to the patterns
 *   - link response y_ij ..................... Eq. (instrument-response-to-gw); n_12 points
 *                                            from emitter 2 to receiver 1 (x1 = x2 + L12 n12)
 *   - delay operators and chained delays ..... Sec. "Time-delay interferometry" (D_ij x(t) =
 *                                            x(t - L_ij(t)); chained delays as sums)
 *   - TDI X1, X2; Y, Z by cyclic permutation . Eqs. (tdi1), (tdi2)
 *   - centered Lagrange interpolation ......... Sec. "Implementation"
 *   - orbit interpolation ..................... Sec. "Implementation" (orbits interpolated
 *                                            to the sample grid): cubic spline
 *   - A, E, T channels ....................... Sec. "Time-delay interferometry" (the
 *                                            uncorrelated combinations of X, Y, Z)
 *   - likelihood inner products .............. Eq. (like), summed over A, E, T, in the time
 *                                            domain with white noise per channel
 * Readings where the paper is silent (order = polynomial degree p, odd; stencil
 * m-(p-1)/2 .. m+(p+1)/2 around m = floor(x); zero extension outside the supplied
 * samples; integer sample index kept exact in read positions; Newtonian light-time solve
 * when delays are not given; nested delays as an option) are the documented readings of the
 * library.
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py (closed forms,
 * invariants, library routines, brute force), except the whole pipeline on generic
 * flexing orbits, which is pinned only through those invariants.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_C 299792458.0
#define ORC_MAX_T 128
#define ORC_NSERIES 15 /* 9 position components + 6 delays */

/* link order used throughout: 12, 23, 31, 13, 32, 21  (receiver, emitter) */
static const int ORC_LINK_R[6] = {1, 2, 3, 1, 3, 2};
static const int ORC_LINK_S[6] = {2, 3, 1, 3, 2, 1};

static int orc_link_index(int r, int s)
{
    for (int l = 0; l < 6; ++l)
        if (ORC_LINK_R[l] == r && ORC_LINK_S[l] == s) return l;
    return -1;
}

/* ------------------------------------------------------------------ threads */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------ Lagrange */
/* Weights of the centered Lagrange interpolating polynomial of degree p (odd) through the
 * nodes j = -(p-1)/2 .. (p+1)/2, evaluated at eps: w_j = prod_{i != j} (eps - i)/(j - i).
 * Direct products, one weight at a time. */
void orc_lagrange_weights(int p, double eps, double *w)
{
    int h = (p - 1) / 2, T = p + 1;
    for (int a = 0; a < T; ++a) {
        int ja = a - h;
        double prod = 1.0;
        for (int b = 0; b < T; ++b) {
            if (b == a) continue;
            int jb = b - h;
            prod *= (eps - (double)jb) / (double)(ja - jb);
        }
        w[a] = prod;
    }
}

/* Derivatives dw_j/deps by the product rule: sum over the factor that is differentiated. */
void orc_lagrange_dweights(int p, double eps, double *dw)
{
    int h = (p - 1) / 2, T = p + 1;
    for (int a = 0; a < T; ++a) {
        int ja = a - h;
        double total = 0.0;
        for (int c = 0; c < T; ++c) {
            if (c == a) continue;
            int jc = c - h;
            double prod = 1.0 / (double)(ja - jc);
            for (int b = 0; b < T; ++b) {
                if (b == a || b == c) continue;
                int jb = b - h;
                prod *= (eps - (double)jb) / (double)(ja - jb);
            }
            total += prod;
        }
        dw[a] = total;
    }
}

/* Value of the series s[0..ns) (zero outside) at fractional sample position base + u:
 * m = base + floor(u), eps = u - floor(u), sum of w_j(eps) s[m + j]. */
double orc_lagrange_read(const double *s, int64_t ns, int64_t base, double u, int p)
{
    double fl = floor(u);
    int64_t m = base + (int64_t)fl;
    double eps = u - fl;
    double w[ORC_MAX_T];
    orc_lagrange_weights(p, eps, w);
    int h = (p - 1) / 2;
    double acc = 0.0;
    for (int a = 0; a < p + 1; ++a) {
        int64_t i = m - h + a;
        if (i >= 0 && i < ns) acc += w[a] * s[i];
    }
    return acc;
}

/* Derivative of the interpolant with respect to the sample position. */
static double orc_lagrange_dread(const double *s, int64_t ns, int64_t base, double u, int p)
{
    double fl = floor(u);
    int64_t m = base + (int64_t)fl;
    double eps = u - fl;
    double dw[ORC_MAX_T];
    orc_lagrange_dweights(p, eps, dw);
    int h = (p - 1) / 2;
    double acc = 0.0;
    for (int a = 0; a < p + 1; ++a) {
        int64_t i = m - h + a;
        if (i >= 0 && i < ns) acc += dw[a] * s[i];
    }
    return acc;
}

/* Same stencil with |w_j| and |s|: the scale of the rounding error of a read. */
static double orc_lagrange_read_abs(const double *s, int64_t ns, int64_t base, double u, int p)
{
    double fl = floor(u);
    int64_t m = base + (int64_t)fl;
    double eps = u - fl;
    double w[ORC_MAX_T];
    orc_lagrange_weights(p, eps, w);
    int h = (p - 1) / 2;
    double acc = 0.0;
    for (int a = 0; a < p + 1; ++a) {
        int64_t i = m - h + a;
        if (i >= 0 && i < ns) acc += fabs(w[a]) * fabs(s[i]);
    }
    return acc;
}

/* ------------------------------------------------------------------ cubic spline */
/* Second derivatives M of the cubic spline through (t_k, y_k), k = 0..n-1 (any spacing).
 * bc = 0: not-a-knot (third derivative continuous at t_1 and t_{n-2});
 * bc = 1: natural (M_0 = M_{n-1} = 0).
 * The n x n system is assembled densely and solved by Gaussian elimination with partial
 * pivoting.  Returns 0 on success. */
static int orc_spline_M(const double *t, const double *y, int64_t n, int bc, double *M)
{
    if (n < 2) return -1;
    if (bc == 0 && n < 4) return -1;
    double *A = (double *)calloc((size_t)(n * n), sizeof(double));
    double *r = (double *)calloc((size_t)n, sizeof(double));
    if (!A || !r) { free(A); free(r); return -2; }
#define AA(i, j) A[(i) * n + (j)]
    if (bc == 1 || n == 2) {
        AA(0, 0) = 1.0; r[0] = 0.0;
        AA(n - 1, n - 1) = 1.0; r[n - 1] = 0.0;
    } else {
        double h0 = t[1] - t[0], h1 = t[2] - t[1];
        AA(0, 0) = h1; AA(0, 1) = -(h0 + h1); AA(0, 2) = h0; r[0] = 0.0;
        double ha = t[n - 2] - t[n - 3], hb = t[n - 1] - t[n - 2];
        AA(n - 1, n - 3) = hb; AA(n - 1, n - 2) = -(ha + hb); AA(n - 1, n - 1) = ha; r[n - 1] = 0.0;
    }
    for (int64_t k = 1; k < n - 1; ++k) {
        double hm = t[k] - t[k - 1], hp = t[k + 1] - t[k];
        AA(k, k - 1) = hm;
        AA(k, k) = 2.0 * (hm + hp);
        AA(k, k + 1) = hp;
        r[k] = 6.0 * ((y[k + 1] - y[k]) / hp - (y[k] - y[k - 1]) / hm);
    }
    /* elimination with partial pivoting */
    for (int64_t c = 0; c < n; ++c) {
        int64_t piv = c;
        for (int64_t i = c + 1; i < n; ++i)
            if (fabs(AA(i, c)) > fabs(AA(piv, c))) piv = i;
        if (AA(piv, c) == 0.0) { free(A); free(r); return -3; }
        if (piv != c) {
            for (int64_t j = 0; j < n; ++j) { double tmp = AA(c, j); AA(c, j) = AA(piv, j); AA(piv, j) = tmp; }
            double tmp = r[c]; r[c] = r[piv]; r[piv] = tmp;
        }
        for (int64_t i = c + 1; i < n; ++i) {
            double f = AA(i, c) / AA(c, c);
            if (f == 0.0) continue;
            for (int64_t j = c; j < n; ++j) AA(i, j) -= f * AA(c, j);
            r[i] -= f * r[c];
        }
    }
    for (int64_t i = n - 1; i >= 0; --i) {
        double s = r[i];
        for (int64_t j = i + 1; j < n; ++j) s -= AA(i, j) * M[j];
        M[i] = s / AA(i, i);
    }
#undef AA
    free(A);
    free(r);
    return 0;
}

/* Spline value at t; outside the knots the first / last cubic piece is continued. */
static double orc_spline_value(const double *tk, const double *y, const double *M, int64_t n, double t)
{
    int64_t lo = 0, hi = n - 1;
    if (t <= tk[0]) { lo = 0; }
    else if (t >= tk[n - 1]) { lo = n - 2; }
    else {
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) / 2;
            if (tk[mid] <= t) lo = mid; else hi = mid;
        }
    }
    if (lo > n - 2) lo = n - 2;
    int64_t k = lo;
    double h = tk[k + 1] - tk[k];
    double A = (tk[k + 1] - t) / h, B = (t - tk[k]) / h;
    return A * y[k] + B * y[k + 1] + ((A * A * A - A) * M[k] + (B * B * B - B) * M[k + 1]) * h * h / 6.0;
}

/* One series, for the tests: spline through (tk, y) evaluated at t[0..nt). */
int orc_spline_eval_series(const double *tk, int64_t nk, const double *y, int bc,
                           const double *t, int64_t nt, double *out)
{
    double *M = (double *)malloc(sizeof(double) * (size_t)nk);
    if (!M) return -2;
    int st = orc_spline_M(tk, y, nk, bc, M);
    if (st) { free(M); return st; }
    for (int64_t i = 0; i < nt; ++i) out[i] = orc_spline_value(tk, y, M, nk, t[i]);
    free(M);
    return 0;
}

/* ------------------------------------------------------------------ orbits */
typedef struct {
    int64_t nk;
    int bc;
    double *tk;      /* [nk] */
    double *val;     /* [15][nk]: x1,y1,z1,x2,..,z3, L12,L23,L31,L13,L32,L21 */
    double *M;       /* [15][nk] second derivatives */
} orc_orbit;

static void orc_orbit_positions(const orc_orbit *o, double t, double x[3][3])
{
    for (int i = 0; i < 3; ++i)
        for (int d = 0; d < 3; ++d) {
            int s = 3 * i + d;
            x[i][d] = orc_spline_value(o->tk, o->val + s * o->nk, o->M + s * o->nk, o->nk, t);
        }
}

static double orc_orbit_delay(const orc_orbit *o, int link, double t)
{
    int s = 9 + link;
    return orc_spline_value(o->tk, o->val + s * o->nk, o->M + s * o->nk, o->nk, t);
}

void orc_orbit_free(void *h)
{
    orc_orbit *o = (orc_orbit *)h;
    if (!o) return;
    free(o->tk); free(o->val); free(o->M); free(o);
}

/* pos: [3 spacecraft][3 xyz][nk] in m.  delays: [6 links][nk] in s, or NULL, in which
 * case each delay on the knots solves the Newtonian light-time equation
 *   L_rs(t) = | x_r(t) - x_s(t - L_rs(t)) | / c
 * (receiver r at reception time t, emitter s at emission time) by fixed-point iteration,
 * with x_s evaluated from the position spline.  The delays are then splined like the
 * positions. */
void *orc_orbit_new(const double *tk, int64_t nk, const double *pos, const double *delays, int bc, int *status)
{
    *status = 0;
    orc_orbit *o = (orc_orbit *)calloc(1, sizeof(orc_orbit));
    if (!o) { *status = -2; return NULL; }
    o->nk = nk; o->bc = bc;
    o->tk = (double *)malloc(sizeof(double) * (size_t)nk);
    o->val = (double *)malloc(sizeof(double) * (size_t)(ORC_NSERIES * nk));
    o->M = (double *)malloc(sizeof(double) * (size_t)(ORC_NSERIES * nk));
    if (!o->tk || !o->val || !o->M) { orc_orbit_free(o); *status = -2; return NULL; }
    memcpy(o->tk, tk, sizeof(double) * (size_t)nk);
    memcpy(o->val, pos, sizeof(double) * (size_t)(9 * nk));
    for (int s = 0; s < 9; ++s) {
        int st = orc_spline_M(o->tk, o->val + s * nk, nk, bc, o->M + s * nk);
        if (st) { orc_orbit_free(o); *status = st; return NULL; }
    }
    if (delays) {
        memcpy(o->val + 9 * nk, delays, sizeof(double) * (size_t)(6 * nk));
    } else {
        for (int l = 0; l < 6; ++l) {
            int r = ORC_LINK_R[l] - 1, s = ORC_LINK_S[l] - 1;
            for (int64_t k = 0; k < nk; ++k) {
                double t = o->tk[k];
                double xr[3], xs[3], x[3][3];
                orc_orbit_positions(o, t, x);
                for (int d = 0; d < 3; ++d) { xr[d] = x[r][d]; xs[d] = x[s][d]; }
                double L = sqrt((xr[0] - xs[0]) * (xr[0] - xs[0]) + (xr[1] - xs[1]) * (xr[1] - xs[1]) +
                                (xr[2] - xs[2]) * (xr[2] - xs[2])) / ORC_C;
                for (int it = 0; it < 100; ++it) {
                    orc_orbit_positions(o, t - L, x);
                    double dx = xr[0] - x[s][0], dy = xr[1] - x[s][1], dz = xr[2] - x[s][2];
                    double Ln = sqrt(dx * dx + dy * dy + dz * dz) / ORC_C;
                    double change = fabs(Ln - L);
                    L = Ln;
                    if (change <= 1e-15 * L) break;
                }
                o->val[(9 + l) * nk + k] = L;
            }
        }
    }
    for (int s = 9; s < ORC_NSERIES; ++s) {
        int st = orc_spline_M(o->tk, o->val + s * nk, nk, bc, o->M + s * nk);
        if (st) { orc_orbit_free(o); *status = st; return NULL; }
    }
    return o;
}

/* positions [9] (x1 y1 z1 x2 .. z3) and delays [6] at time t */
void orc_orbit_eval(const void *h, double t, double *pos9, double *del6)
{
    const orc_orbit *o = (const orc_orbit *)h;
    double x[3][3];
    orc_orbit_positions(o, t, x);
    for (int i = 0; i < 3; ++i)
        for (int d = 0; d < 3; ++d) pos9[3 * i + d] = x[i][d];
    for (int l = 0; l < 6; ++l) del6[l] = orc_orbit_delay(o, l, t);
}

void orc_orbit_delays_at_knots(const void *h, double *out)
{
    const orc_orbit *o = (const orc_orbit *)h;
    memcpy(out, o->val + 9 * o->nk, sizeof(double) * (size_t)(6 * o->nk));
}

/* ------------------------------------------------------------------ sky frame */
/* e_r = (cos b cos l, cos b sin l, sin b), e_theta = (sin b cos l, sin b sin l, -cos b),
 * e_phi = (-sin l, cos l, 0); k = -e_r, u = -e_phi, v = -e_theta.  Also returns the
 * derivatives of k, u, v with respect to lambda and beta. */
typedef struct {
    double k[3], u[3], v[3];
    double dk_dl[3], du_dl[3], dv_dl[3];
    double dk_db[3], du_db[3], dv_db[3];
    double c2p, s2p;
} orc_sky;

void orc_sky_basis(double lam, double beta, double *k, double *u, double *v)
{
    double cl = cos(lam), sl = sin(lam), cb = cos(beta), sb = sin(beta);
    double er[3] = {cb * cl, cb * sl, sb};
    double et[3] = {sb * cl, sb * sl, -cb};
    double ep[3] = {-sl, cl, 0.0};
    for (int d = 0; d < 3; ++d) { k[d] = -er[d]; u[d] = -ep[d]; v[d] = -et[d]; }
}

static void orc_sky_make(double lam, double beta, double psi, orc_sky *S)
{
    double cl = cos(lam), sl = sin(lam), cb = cos(beta), sb = sin(beta);
    orc_sky_basis(lam, beta, S->k, S->u, S->v);
    double der_dl[3] = {-cb * sl, cb * cl, 0.0}, der_db[3] = {-sb * cl, -sb * sl, cb};
    double det_dl[3] = {-sb * sl, sb * cl, 0.0}, det_db[3] = {cb * cl, cb * sl, sb};
    double dep_dl[3] = {-cl, -sl, 0.0}, dep_db[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < 3; ++d) {
        S->dk_dl[d] = -der_dl[d]; S->dk_db[d] = -der_db[d];
        S->du_dl[d] = -dep_dl[d]; S->du_db[d] = -dep_db[d];
        S->dv_dl[d] = -det_dl[d]; S->dv_db[d] = -det_db[d];
    }
    S->c2p = cos(2.0 * psi);
    S->s2p = sin(2.0 * psi);
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ------------------------------------------------------------------ geometry of one link */
typedef struct {
    double n[3];         /* unit vector from emitter to receiver */
    double xp, xc;       /* psi-rotated antenna patterns */
    double kn;           /* k . n */
    double ur, ue;       /* read positions (sample units, relative to the integer base) */
} orc_link_geo;

/* Geometry of link l at output sample n (time t = t0 + n dt) from positions x and delays L.
 * Read positions in the h grid (t0_h + j dt): receiver (t - k.x_r/c - t0_h)/dt and emitter
 * (t - L_l - k.x_s/c - t0_h)/dt, written as n + u with the integer n kept exact. */
static void orc_link_geometry(int l, const double x[3][3], const double *L, const orc_sky *S,
                              double t0, double dt, double t0h, orc_link_geo *g)
{
    int r = ORC_LINK_R[l] - 1, s = ORC_LINK_S[l] - 1;
    double d[3] = {x[r][0] - x[s][0], x[r][1] - x[s][1], x[r][2] - x[s][2]};
    double norm = sqrt(dot3(d, d));
    for (int c = 0; c < 3; ++c) g->n[c] = d[c] / norm;
    double a = dot3(S->u, g->n), b = dot3(S->v, g->n);
    double xip = a * a - b * b, xic = 2.0 * a * b;
    g->xp = S->c2p * xip + S->s2p * xic;
    g->xc = -S->s2p * xip + S->c2p * xic;
    g->kn = dot3(S->k, g->n);
    double u0 = (t0 - t0h) / dt;
    g->ur = u0 - dot3(S->k, x[r]) / ORC_C / dt;
    g->ue = u0 - L[l] / dt - dot3(S->k, x[s]) / ORC_C / dt;
}

/* ------------------------------------------------------------------ projection */
/* y_l(t_n) = [H_l(t - L_l - k.x_s/c) - H_l(t - k.x_r/c)] / (2 (1 - k.n_l)),
 * H_l(tau) = xi+_l h+(tau) + xix_l hx(tau); zero for n outside [0, N). */
static void orc_y_at(int p, double dt, double t0, int64_t N, const orc_orbit *po,
                     const double *hp, const double *hc, int64_t nh, double t0h,
                     const orc_sky *S, int64_t n, double y[6])
{
    if (n < 0 || n >= N) { for (int l = 0; l < 6; ++l) y[l] = 0.0; return; }
    double t = t0 + (double)n * dt;
    double x[3][3], L[6];
    orc_orbit_positions(po, t, x);
    for (int l = 0; l < 6; ++l) L[l] = orc_orbit_delay(po, l, t);
    for (int l = 0; l < 6; ++l) {
        orc_link_geo g;
        orc_link_geometry(l, x, L, S, t0, dt, t0h, &g);
        double He = g.xp * orc_lagrange_read(hp, nh, n, g.ue, p) + g.xc * orc_lagrange_read(hc, nh, n, g.ue, p);
        double Hr = g.xp * orc_lagrange_read(hp, nh, n, g.ur, p) + g.xc * orc_lagrange_read(hc, nh, n, g.ur, p);
        y[l] = (He - Hr) / (2.0 * (1.0 - g.kn));
    }
}

/* absolute-value version: the scale of the rounding error of y */
static void orc_y_abs_at(int p, double dt, double t0, int64_t N, const orc_orbit *po,
                         const double *hp, const double *hc, int64_t nh, double t0h,
                         const orc_sky *S, int64_t n, double y[6])
{
    if (n < 0 || n >= N) { for (int l = 0; l < 6; ++l) y[l] = 0.0; return; }
    double t = t0 + (double)n * dt;
    double x[3][3], L[6];
    orc_orbit_positions(po, t, x);
    for (int l = 0; l < 6; ++l) L[l] = orc_orbit_delay(po, l, t);
    for (int l = 0; l < 6; ++l) {
        orc_link_geo g;
        orc_link_geometry(l, x, L, S, t0, dt, t0h, &g);
        double He = fabs(g.xp) * orc_lagrange_read_abs(hp, nh, n, g.ue, p) +
                    fabs(g.xc) * orc_lagrange_read_abs(hc, nh, n, g.ue, p);
        double Hr = fabs(g.xp) * orc_lagrange_read_abs(hp, nh, n, g.ur, p) +
                    fabs(g.xc) * orc_lagrange_read_abs(hc, nh, n, g.ur, p);
        y[l] = (He + Hr) / fabs(2.0 * (1.0 - g.kn));
    }
}

int orc_project(int p, double dt, double t0, int64_t N, const void *porb,
                const double *hp, const double *hc, int64_t nh, double t0h,
                double lam, double beta, double psi, double *y)
{
    if (p < 1 || (p % 2) == 0 || p + 1 > ORC_MAX_T) return -1;
    orc_sky S;
    orc_sky_make(lam, beta, psi, &S);
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double v[6];
        orc_y_at(p, dt, t0, N, (const orc_orbit *)porb, hp, hc, nh, t0h, &S, n, v);
        for (int l = 0; l < 6; ++l) y[(int64_t)l * N + n] = v[l];
    }
    return 0;
}

int orc_project_abs(int p, double dt, double t0, int64_t N, const void *porb,
                    const double *hp, const double *hc, int64_t nh, double t0h,
                    double lam, double beta, double psi, double *y)
{
    if (p < 1 || (p % 2) == 0 || p + 1 > ORC_MAX_T) return -1;
    orc_sky S;
    orc_sky_make(lam, beta, psi, &S);
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double v[6];
        orc_y_abs_at(p, dt, t0, N, (const orc_orbit *)porb, hp, hc, nh, t0h, &S, n, v);
        for (int l = 0; l < 6; ++l) y[(int64_t)l * N + n] = v[l];
    }
    return 0;
}

/* ------------------------------------------------------------------ TDI */
/* The Michelson combinations exactly as printed: each term is (sign, delay indices, link).
 * X1 is the first 8 terms, X2 all 16. */
typedef struct { int sign; const char *delay; const char *link; } orc_term;
static const orc_term ORC_X2[16] = {
    {+1, "", "13"}, {+1, "13", "31"}, {+1, "131", "12"}, {+1, "1312", "21"},
    {-1, "", "12"}, {-1, "12", "21"}, {-1, "121", "13"}, {-1, "1213", "31"},
    {+1, "13121", "12"}, {+1, "131212", "21"}, {+1, "1312121", "13"}, {+1, "13121213", "31"},
    {-1, "12131", "13"}, {-1, "121313", "31"}, {-1, "1213131", "12"}, {-1, "12131312", "21"},
};

/* cyclic permutation 1 -> 2 -> 3 -> 1 applied `times` times to a spacecraft index */
static int orc_perm(int i, int times)
{
    for (int k = 0; k < times; ++k) i = (i % 3) + 1;
    return i;
}

/* Total delay (s) of the chained operator D_{i1 i2 .. in} at time t for channel `ch`
 * (0 = X, 1 = Y, 2 = Z).  delay_mode 0: sum of L_{i_k i_{k+1}}(t) (the paper's choice);
 * delay_mode 1: nested, t_1 = t - L_{i1 i2}(t), t_2 = t_1 - L_{i2 i3}(t_1), ... */
static double orc_chain_delay(const orc_orbit *to, const char *idx, int ch, int delay_mode, double t)
{
    int len = (int)strlen(idx);
    if (len < 2) return 0.0;
    if (delay_mode == 0) {
        double D = 0.0;
        for (int k = 0; k + 1 < len; ++k) {
            int a = orc_perm(idx[k] - '0', ch), b = orc_perm(idx[k + 1] - '0', ch);
            D += orc_orbit_delay(to, orc_link_index(a, b), t);
        }
        return D;
    }
    double tc = t;
    for (int k = 0; k + 1 < len; ++k) {
        int a = orc_perm(idx[k] - '0', ch), b = orc_perm(idx[k + 1] - '0', ch);
        tc = tc - orc_orbit_delay(to, orc_link_index(a, b), tc);
    }
    return t - tc;
}

static int orc_term_link(const char *link, int ch)
{
    return orc_link_index(orc_perm(link[0] - '0', ch), orc_perm(link[1] - '0', ch));
}

/* X, Y, Z at output sample n from the six link series y[6][N] (zero outside [0, N)) */
static void orc_xyz_at(int p, int gen, int delay_mode, double dt, double t0, int64_t N,
                       const orc_orbit *to, const double *y, int64_t n, double out[3], int absval)
{
    double t = t0 + (double)n * dt;
    int nterms = gen == 1 ? 8 : 16;
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
        for (int q = 0; q < nterms; ++q) {
            const orc_term *tm = &ORC_X2[q];
            int l = orc_term_link(tm->link, ch);
            double D = orc_chain_delay(to, tm->delay, ch, delay_mode, t);
            double v = absval ? orc_lagrange_read_abs(y + (int64_t)l * N, N, n, -D / dt, p)
                              : orc_lagrange_read(y + (int64_t)l * N, N, n, -D / dt, p);
            acc += absval ? v : (double)tm->sign * v;
        }
        out[ch] = acc;
    }
}

int orc_tdi(int p, int gen, int delay_mode, double dt, double t0, int64_t N, const void *torb,
            const double *y, double *xyz)
{
    if (p < 1 || (p % 2) == 0 || p + 1 > ORC_MAX_T || (gen != 1 && gen != 2)) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double v[3];
        orc_xyz_at(p, gen, delay_mode, dt, t0, N, (const orc_orbit *)torb, y, n, v, 0);
        for (int c = 0; c < 3; ++c) xyz[(int64_t)c * N + n] = v[c];
    }
    return 0;
}

/* error scale of the TDI stage: |w| applied to the error scale of y */
int orc_tdi_abs(int p, int gen, int delay_mode, double dt, double t0, int64_t N, const void *torb,
                const double *yabs, double *xyz)
{
    if (p < 1 || (p % 2) == 0 || p + 1 > ORC_MAX_T || (gen != 1 && gen != 2)) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double v[3];
        orc_xyz_at(p, gen, delay_mode, dt, t0, N, (const orc_orbit *)torb, yabs, n, v, 1);
        for (int c = 0; c < 3; ++c) xyz[(int64_t)c * N + n] = v[c];
    }
    return 0;
}

/* X, Y, Z at a list of output indices, computing y on demand around each index (for long
 * series where the full y would be too slow to build). */
int orc_response_at(int p, int gen, int delay_mode, double dt, double t0, int64_t N,
                    const void *porb, const void *torb,
                    const double *hp, const double *hc, int64_t nh, double t0h,
                    double lam, double beta, double psi,
                    const int64_t *idx, int64_t nidx, double *xyz, int absval)
{
    if (p < 1 || (p % 2) == 0 || p + 1 > ORC_MAX_T || (gen != 1 && gen != 2)) return -1;
    const orc_orbit *po = (const orc_orbit *)porb, *to = (const orc_orbit *)torb;
    orc_sky S;
    orc_sky_make(lam, beta, psi, &S);
    int h = (p - 1) / 2;
    int nterms = gen == 1 ? 8 : 16;
    int status = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nidx; ++q) {
        int64_t n = idx[q];
        double t = t0 + (double)n * dt;
        /* the furthest delayed read reaches back by the largest chain delay */
        double Dmax = 0.0;
        for (int ch = 0; ch < 3; ++ch)
            for (int k = 0; k < nterms; ++k) {
                double D = orc_chain_delay(to, ORC_X2[k].delay, ch, delay_mode, t);
                if (D > Dmax) Dmax = D;
            }
        int64_t lo = n - (int64_t)ceil(Dmax / dt) - h - 2, hi = n + h + 2;
        int64_t W = hi - lo + 1;
        double *win = (double *)malloc(sizeof(double) * (size_t)(6 * W));
        if (!win) { status = -2; continue; }
        for (int64_t k = lo; k <= hi; ++k) {
            double v[6];
            if (absval) orc_y_abs_at(p, dt, t0, N, po, hp, hc, nh, t0h, &S, k, v);
            else orc_y_at(p, dt, t0, N, po, hp, hc, nh, t0h, &S, k, v);
            for (int l = 0; l < 6; ++l) win[(int64_t)l * W + (k - lo)] = v[l];
        }
        /* the window holds y[lo..hi]; reads outside it are outside the stencil reach */
        for (int ch = 0; ch < 3; ++ch) {
            double acc = 0.0;
            for (int k = 0; k < nterms; ++k) {
                const orc_term *tm = &ORC_X2[k];
                int l = orc_term_link(tm->link, ch);
                double D = orc_chain_delay(to, tm->delay, ch, delay_mode, t);
                double v = absval ? orc_lagrange_read_abs(win + (int64_t)l * W, W, n - lo, -D / dt, p)
                                  : orc_lagrange_read(win + (int64_t)l * W, W, n - lo, -D / dt, p);
                acc += absval ? v : (double)tm->sign * v;
            }
            xyz[(int64_t)ch * nidx + q] = acc;
        }
        free(win);
    }
    return status;
}

/* y at a list of output indices */
int orc_project_at(int p, double dt, double t0, int64_t N, const void *porb,
                   const double *hp, const double *hc, int64_t nh, double t0h,
                   double lam, double beta, double psi, const int64_t *idx, int64_t nidx, double *y)
{
    if (p < 1 || (p % 2) == 0 || p + 1 > ORC_MAX_T) return -1;
    orc_sky S;
    orc_sky_make(lam, beta, psi, &S);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < nidx; ++q) {
        double v[6];
        orc_y_at(p, dt, t0, N, (const orc_orbit *)porb, hp, hc, nh, t0h, &S, idx[q], v);
        for (int l = 0; l < 6; ++l) y[(int64_t)l * nidx + q] = v[l];
    }
    return 0;
}

/* ------------------------------------------------------------------ adjoints */
/* Transpose of the TDI stage by explicit scatter: every tap of every term of every output
 * adds its weight times the incoming gradient into the link sample it read. */
int orc_tdi_adjoint(int p, int gen, int delay_mode, double dt, double t0, int64_t N, const void *torb,
                    const double *gxyz, double *gy)
{
    if (p < 1 || (p % 2) == 0 || p + 1 > ORC_MAX_T || (gen != 1 && gen != 2)) return -1;
    const orc_orbit *to = (const orc_orbit *)torb;
    int h = (p - 1) / 2;
    int nterms = gen == 1 ? 8 : 16;
    memset(gy, 0, sizeof(double) * (size_t)(6 * N));
    double w[ORC_MAX_T];
    for (int64_t n = 0; n < N; ++n) {
        double t = t0 + (double)n * dt;
        for (int ch = 0; ch < 3; ++ch) {
            double g = gxyz[(int64_t)ch * N + n];
            for (int k = 0; k < nterms; ++k) {
                const orc_term *tm = &ORC_X2[k];
                int l = orc_term_link(tm->link, ch);
                double D = orc_chain_delay(to, tm->delay, ch, delay_mode, t);
                double u = -D / dt, fl = floor(u);
                int64_t m = n + (int64_t)fl;
                orc_lagrange_weights(p, u - fl, w);
                for (int a = 0; a < p + 1; ++a) {
                    int64_t i = m - h + a;
                    if (i >= 0 && i < N) gy[(int64_t)l * N + i] += (double)tm->sign * w[a] * g;
                }
            }
        }
    }
    return 0;
}

/* Transpose of the projection by explicit scatter into g_h+, g_hx. */
int orc_project_adjoint(int p, double dt, double t0, int64_t N, const void *porb, int64_t nh, double t0h,
                        double lam, double beta, double psi, const double *gy, double *ghp, double *ghc)
{
    if (p < 1 || (p % 2) == 0 || p + 1 > ORC_MAX_T) return -1;
    const orc_orbit *po = (const orc_orbit *)porb;
    orc_sky S;
    orc_sky_make(lam, beta, psi, &S);
    int h = (p - 1) / 2;
    memset(ghp, 0, sizeof(double) * (size_t)nh);
    memset(ghc, 0, sizeof(double) * (size_t)nh);
    double w[ORC_MAX_T];
    for (int64_t n = 0; n < N; ++n) {
        double t = t0 + (double)n * dt;
        double x[3][3], L[6];
        orc_orbit_positions(po, t, x);
        for (int l = 0; l < 6; ++l) L[l] = orc_orbit_delay(po, l, t);
        for (int l = 0; l < 6; ++l) {
            orc_link_geo g;
            orc_link_geometry(l, x, L, &S, t0, dt, t0h, &g);
            double c = gy[(int64_t)l * N + n] / (2.0 * (1.0 - g.kn));
            for (int side = 0; side < 2; ++side) {
                double u = side == 0 ? g.ue : g.ur, sgn = side == 0 ? 1.0 : -1.0;
                double fl = floor(u);
                int64_t m = n + (int64_t)fl;
                orc_lagrange_weights(p, u - fl, w);
                for (int a = 0; a < p + 1; ++a) {
                    int64_t i = m - h + a;
                    if (i < 0 || i >= nh) continue;
                    ghp[i] += sgn * c * g.xp * w[a];
                    ghc[i] += sgn * c * g.xc * w[a];
                }
            }
        }
    }
    return 0;
}

/* dLoss/d(lambda, beta, psi) = sum_n sum_l g_y[l][n] dy_l[n]/dtheta, with
 * dy = d(1/(2(1 - k.n))) * dH + (1/(2(1 - k.n))) * d(dH), where dH = H(tau_e) - H(tau_r)
 * changes through the patterns and through the read times tau = t - ... - k.x/c. */
int orc_sky_gradient(int p, double dt, double t0, int64_t N, const void *porb,
                     const double *hp, const double *hc, int64_t nh, double t0h,
                     double lam, double beta, double psi, const double *gy, double *gsky)
{
    if (p < 1 || (p % 2) == 0 || p + 1 > ORC_MAX_T) return -1;
    const orc_orbit *po = (const orc_orbit *)porb;
    orc_sky S;
    orc_sky_make(lam, beta, psi, &S);
    double G[3] = {0.0, 0.0, 0.0};
    for (int64_t n = 0; n < N; ++n) {
        double t = t0 + (double)n * dt;
        double x[3][3], L[6];
        orc_orbit_positions(po, t, x);
        for (int l = 0; l < 6; ++l) L[l] = orc_orbit_delay(po, l, t);
        for (int l = 0; l < 6; ++l) {
            double gl = gy[(int64_t)l * N + n];
            if (gl == 0.0) continue;
            int r = ORC_LINK_R[l] - 1, s = ORC_LINK_S[l] - 1;
            orc_link_geo g;
            orc_link_geometry(l, x, L, &S, t0, dt, t0h, &g);
            double den = 1.0 / (2.0 * (1.0 - g.kn));
            double Pe_p = orc_lagrange_read(hp, nh, n, g.ue, p), Pr_p = orc_lagrange_read(hp, nh, n, g.ur, p);
            double Pe_c = orc_lagrange_read(hc, nh, n, g.ue, p), Pr_c = orc_lagrange_read(hc, nh, n, g.ur, p);
            double dPe_p = orc_lagrange_dread(hp, nh, n, g.ue, p), dPr_p = orc_lagrange_dread(hp, nh, n, g.ur, p);
            double dPe_c = orc_lagrange_dread(hc, nh, n, g.ue, p), dPr_c = orc_lagrange_dread(hc, nh, n, g.ur, p);
            double dH = g.xp * (Pe_p - Pr_p) + g.xc * (Pe_c - Pr_c);
            double a = dot3(S.u, g.n), b = dot3(S.v, g.n);
            double xip = a * a - b * b, xic = 2.0 * a * b;
            for (int th = 0; th < 2; ++th) {
                const double *dk = th == 0 ? S.dk_dl : S.dk_db;
                const double *du = th == 0 ? S.du_dl : S.du_db;
                const double *dv = th == 0 ? S.dv_dl : S.dv_db;
                double da = dot3(du, g.n), db = dot3(dv, g.n);
                double dxip = 2.0 * a * da - 2.0 * b * db, dxic = 2.0 * (da * b + a * db);
                double dxp = S.c2p * dxip + S.s2p * dxic, dxc = -S.s2p * dxip + S.c2p * dxic;
                double dden = 2.0 * den * den * dot3(dk, g.n);
                double due = -dot3(dk, x[s]) / ORC_C / dt, dur = -dot3(dk, x[r]) / ORC_C / dt;
                double ddH = dxp * (Pe_p - Pr_p) + dxc * (Pe_c - Pr_c) +
                             g.xp * (dPe_p * due - dPr_p * dur) + g.xc * (dPe_c * due - dPr_c * dur);
                G[th] += gl * (dden * dH + den * ddH);
            }
            /* psi: d xp/dpsi = 2 xc, d xc/dpsi = -2 xp */
            double ddHpsi = 2.0 * g.xc * (Pe_p - Pr_p) - 2.0 * g.xp * (Pe_c - Pr_c);
            G[2] += gl * den * ddHpsi;
        }
    }
    gsky[0] = G[0]; gsky[1] = G[1]; gsky[2] = G[2];
    return 0;
}

/* Rounding-error scale of the sky-angle gradient: the same sums with every factor replaced by
 * its absolute value (reads with |w| and |w'|).  Used only to size test tolerances. */
static double orc_lagrange_dread_abs(const double *s, int64_t ns, int64_t base, double u, int p)
{
    double fl = floor(u);
    int64_t m = base + (int64_t)fl;
    double eps = u - fl;
    double dw[ORC_MAX_T];
    orc_lagrange_dweights(p, eps, dw);
    int h = (p - 1) / 2;
    double acc = 0.0;
    for (int a = 0; a < p + 1; ++a) {
        int64_t i = m - h + a;
        if (i >= 0 && i < ns) acc += fabs(dw[a]) * fabs(s[i]);
    }
    return acc;
}

int orc_sky_gradient_abs(int p, double dt, double t0, int64_t N, const void *porb,
                         const double *hp, const double *hc, int64_t nh, double t0h,
                         double lam, double beta, double psi, const double *gy, double *gsky)
{
    if (p < 1 || (p % 2) == 0 || p + 1 > ORC_MAX_T) return -1;
    const orc_orbit *po = (const orc_orbit *)porb;
    orc_sky S;
    orc_sky_make(lam, beta, psi, &S);
    double G[3] = {0.0, 0.0, 0.0};
    for (int64_t n = 0; n < N; ++n) {
        double t = t0 + (double)n * dt;
        double x[3][3], L[6];
        orc_orbit_positions(po, t, x);
        for (int l = 0; l < 6; ++l) L[l] = orc_orbit_delay(po, l, t);
        for (int l = 0; l < 6; ++l) {
            double gl = fabs(gy[(int64_t)l * N + n]);
            if (gl == 0.0) continue;
            int r = ORC_LINK_R[l] - 1, s = ORC_LINK_S[l] - 1;
            orc_link_geo g;
            orc_link_geometry(l, x, L, &S, t0, dt, t0h, &g);
            double den = fabs(1.0 / (2.0 * (1.0 - g.kn)));
            double Ap = orc_lagrange_read_abs(hp, nh, n, g.ue, p) + orc_lagrange_read_abs(hp, nh, n, g.ur, p);
            double Ac = orc_lagrange_read_abs(hc, nh, n, g.ue, p) + orc_lagrange_read_abs(hc, nh, n, g.ur, p);
            double dAe_p = orc_lagrange_dread_abs(hp, nh, n, g.ue, p), dAr_p = orc_lagrange_dread_abs(hp, nh, n, g.ur, p);
            double dAe_c = orc_lagrange_dread_abs(hc, nh, n, g.ue, p), dAr_c = orc_lagrange_dread_abs(hc, nh, n, g.ur, p);
            double dH = fabs(g.xp) * Ap + fabs(g.xc) * Ac;
            double a = dot3(S.u, g.n), b = dot3(S.v, g.n);
            for (int th = 0; th < 2; ++th) {
                const double *dk = th == 0 ? S.dk_dl : S.dk_db;
                const double *du = th == 0 ? S.du_dl : S.du_db;
                const double *dv = th == 0 ? S.dv_dl : S.dv_db;
                double da = fabs(dot3(du, g.n)), db = fabs(dot3(dv, g.n));
                double dxi = 2.0 * (fabs(a) * da + fabs(b) * db);
                double dden = 2.0 * den * den * fabs(dot3(dk, g.n));
                double due = fabs(dot3(dk, x[s])) / ORC_C / dt, dur = fabs(dot3(dk, x[r])) / ORC_C / dt;
                double ddH = dxi * (Ap + Ac) + fabs(g.xp) * (dAe_p * due + dAr_p * dur) +
                             fabs(g.xc) * (dAe_c * due + dAr_c * dur);
                G[th] += gl * (dden * dH + den * ddH);
            }
            G[2] += gl * den * 2.0 * (fabs(g.xc) * Ap + fabs(g.xp) * Ac);
        }
    }
    gsky[0] = G[0]; gsky[1] = G[1]; gsky[2] = G[2];
    return 0;
}

/* ------------------------------------------------------------------ Galactic binary */
/* Polarisations of a Galactic binary at t = t0 + j dt, j = 0 .. n-1 (Sec. "Template generation"):
 * the source-frame waveform h+^S = A cos Phi, hx^S = A sin Phi with
 * Phi(t) = 2 pi (f0 t + fdot t^2 / 2 + fddot t^3 / 6) + phi0, weighted by the inclination factors
 * (1 + cos^2 iota) and 2 cos iota of the transform to the SSB frame.  The polarisation angle psi of
 * that transform is applied by the response (the 2 psi rotation of the antenna patterns), and the
 * transform's overall minus sign is the caller's (the library's inputs are the un-rotated
 * polarisations).  fddot is given (the paper takes 11 fdot^2 / (3 f0)). */
void orc_gb_polarisations(double A, double f0, double fdot, double fddot, double phi0, double iota,
                          double t0, double dt, int64_t n, double *hp, double *hc)
{
    const double pi = 4.0 * atan(1.0);
    const double ci = cos(iota);
    for (int64_t j = 0; j < n; ++j) {
        double t = t0 + (double)j * dt;
        double ph = 2.0 * pi * (f0 * t + 0.5 * fdot * t * t + fddot * t * t * t / 6.0) + phi0;
        hp[j] = A * (1.0 + ci * ci) * cos(ph);
        hc[j] = 2.0 * A * ci * sin(ph);
    }
}

/* ------------------------------------------------------------------ likelihood
 * Uncorrelated TDI channels (Sec. "Time-delay interferometry", the A, E, T combinations of
 * X, Y, Z): A = (Z - X)/sqrt(2), E = (X - 2Y + Z)/sqrt(6), T = (X + Y + Z)/sqrt(3).
 * xyz and aet are [3][n] (channel-major). */
void orc_aet(const double *xyz, int64_t n, double *aet)
{
    for (int64_t i = 0; i < n; ++i) {
        const double X = xyz[i], Y = xyz[n + i], Z = xyz[2 * n + i];
        aet[i] = (Z - X) / sqrt(2.0);
        aet[n + i] = (X - 2.0 * Y + Z) / sqrt(6.0);
        aet[2 * n + i] = (X + Y + Z) / sqrt(3.0);
    }
}

/* Inner products of the log-likelihood (Eq. like: log L = -(<d|d> + <h|h> - 2 <d|h>)/2), summed
 * over the channels A, E, T as the paper does, in the time domain with white noise of variance
 * 1/w_c in channel c: <a|b> = sum_c w_c sum_i a_c[i] b_c[i].  The template is given by its
 * X, Y, Z (xyz, [3][n]); the data by its A, E, T (data, [3][n]).  out = {<d|h>, <h|h>}. */
void orc_like_inner(const double *xyz, const double *data, int64_t n, const double *w, double *out)
{
    double *h = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    orc_aet(xyz, n, h);
    double dh = 0.0, hh = 0.0;
    for (int c = 0; c < 3; ++c)
        for (int64_t i = 0; i < n; ++i) {
            dh += w[c] * data[c * n + i] * h[c * n + i];
            hh += w[c] * h[c * n + i] * h[c * n + i];
        }
    free(h);
    out[0] = dh;
    out[1] = hh;
}
