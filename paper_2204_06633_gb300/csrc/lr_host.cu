// Host side of the C ABI: contexts, orbit setup (cubic splines on a uniform knot grid, Newtonian
// light-time solve), plans (halo and window sizing, launch shapes) and argument validation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "lr_internal.h"
#include "lr_bwd.h"
#include "lr_launch.h"
#include "lr_pipeline.h"
#include "lr_planview.h"
#include "lr_tdi_table.cuh"

struct lr_ctx {
    int device;
    int sms;
    int last_cuda_error;
};

struct lr_orbit {
    lr_ctx *ctx;
    int64_t nk;
    int nint;
    double t_first, dk;
    std::vector<double> delays;   // [6][nk], given or solved
    std::vector<double> coef;     // host copy [nint][15][4]
    double *d_coef;
    double max_r_over_c;          // max_t max_i |x_i(t)| / c  (s)
    double max_delay;             // max_t max_l L_l(t)     (s)
    double max_rate;              // bound of |d(k.x_i/c)/dt| + |dL_l/dt| (s/s)
};

struct lr_plan {
    lr_ctx *ctx;
    lr_plan_desc desc;
    lr::FwdParams base;
    int T, h;
    int threads;
    int *d_err;
    int64_t *d_tile_off;
    int64_t tile_cap;
    // backward workspace: link-series gradient, per-tile sky partials, batch tile tables
    double *d_gy;
    int64_t gy_cap;
    double *d_partial;
    int64_t partial_cap;
    int64_t *d_ktile_off, *d_htile_off;
    int64_t ktile_cap;
    // host-buffer pipeline (lr_response_batched_host), created on first use
    lr::PipeWork *pipe;
    // per-tile likelihood partials
    double *d_lpart;
    int64_t lpart_cap;
    // nested-delay table of the mixed kernels ([knots][42], samples)
    double *d_nest;
    // constant-delay TDI weights of the FP64 kernels ([3][2][8][T]), or null
    double *d_cdw;
};

namespace lr {
// Fault injection for tests: after `g_alloc_budget` more successful allocations every further
// library allocation fails as if the device were out of memory (negative: disabled).
static int g_alloc_budget = -1;

cudaError_t dev_malloc(void **p, size_t bytes)
{
    if (g_alloc_budget == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    if (g_alloc_budget > 0) --g_alloc_budget;
    return cudaMalloc(p, bytes);
}
}  // namespace lr

namespace {

int cuda_fail(lr_ctx *ctx, cudaError_t e)
{
    if (ctx) ctx->last_cuda_error = (int)e;
    return e == cudaErrorMemoryAllocation ? LR_ERR_OOM : LR_ERR_CUDA;
}

int check_launch(lr_ctx *ctx, int e)
{
    if (e == 0) return LR_OK;
    return cuda_fail(ctx, (cudaError_t)e);
}

// ---------------------------------------------------------------- spline setup (host)
// Second derivatives M of the interpolating cubic spline on uniform knots (spacing dk):
// interior rows M_{k-1} + 4 M_k + M_{k+1} = 6 (y_{k+1} - 2 y_k + y_{k-1}) / dk^2.
// not-a-knot: M_0 = 2 M_1 - M_2 and M_{n-1} = 2 M_{n-2} - M_{n-3} (third derivative
// continuous at the second and penultimate knots), which turns the first and last interior
// rows into 6 M_1 = rhs_1 and 6 M_{n-2} = rhs_{n-2}; natural: M_0 = M_{n-1} = 0.
// The tridiagonal system is solved by forward elimination and back substitution.
bool spline_second_derivatives(const double *y, int64_t n, double dk, int bc, std::vector<double> &M)
{
    M.assign((size_t)n, 0.0);
    if (n < 3) return n == 2;  // two knots: straight line
    int64_t m = n - 2;         // unknowns M_1 .. M_{n-2}
    std::vector<double> a(m), b(m), c(m), r(m);
    for (int64_t i = 0; i < m; ++i) {
        int64_t k = i + 1;
        a[i] = 1.0; b[i] = 4.0; c[i] = 1.0;
        r[i] = 6.0 * (y[k + 1] - 2.0 * y[k] + y[k - 1]) / (dk * dk);
    }
    if (bc == LR_SPLINE_NOT_A_KNOT) {
        b[0] = 6.0; c[0] = 0.0;
        b[m - 1] = 6.0; a[m - 1] = 0.0;
        if (m == 1) { b[0] = 6.0; }
    }
    a[0] = 0.0;
    c[m - 1] = 0.0;
    for (int64_t i = 1; i < m; ++i) {
        double w = a[i] / b[i - 1];
        b[i] -= w * c[i - 1];
        r[i] -= w * r[i - 1];
    }
    std::vector<double> x(m);
    x[m - 1] = r[m - 1] / b[m - 1];
    for (int64_t i = m - 2; i >= 0; --i) x[i] = (r[i] - c[i] * x[i + 1]) / b[i];
    for (int64_t i = 0; i < m; ++i) M[i + 1] = x[i];
    if (bc == LR_SPLINE_NOT_A_KNOT) {
        if (n < 4) return false;
        M[0] = 2.0 * M[1] - M[2];
        M[n - 1] = 2.0 * M[n - 2] - M[n - 3];
    }
    return true;
}

// Piecewise coefficients in the normalised coordinate x = (t - t_k)/dk:
// S = y_k + b x + c x^2 + d x^3 with b = (y_{k+1}-y_k) - dk^2 (2 M_k + M_{k+1})/6,
// c = dk^2 M_k / 2, d = dk^2 (M_{k+1} - M_k)/6.
void spline_coefficients(const double *y, const std::vector<double> &M, int64_t n, double dk, double *coef,
                         int series)
{
    double h2 = dk * dk;
    for (int64_t k = 0; k + 1 < n; ++k) {
        double *q = coef + ((size_t)k * lr::NSERIES + series) * 4;
        q[0] = y[k];
        q[1] = (y[k + 1] - y[k]) - h2 * (2.0 * M[k] + M[k + 1]) / 6.0;
        q[2] = h2 * M[k] / 2.0;
        q[3] = h2 * (M[k + 1] - M[k]) / 6.0;
    }
}

double spline_eval_host(const lr_orbit *o, int series, double t)
{
    double u = (t - o->t_first) / o->dk;
    int64_t k = (int64_t)std::floor(u);
    if (k < 0) k = 0;
    if (k > o->nint - 1) k = o->nint - 1;
    double x = u - (double)k;
    const double *q = o->coef.data() + ((size_t)k * lr::NSERIES + series) * 4;
    return q[0] + x * (q[1] + x * (q[2] + x * q[3]));
}

const int LINK_R[6] = {0, 1, 2, 0, 2, 1};  // link order 12, 23, 31, 13, 32, 21 (0-based)
const int LINK_S[6] = {1, 2, 0, 2, 1, 0};

// Newtonian light time of link (r <- s) received at t: L = |x_r(t) - x_s(t - L)|/c, solved by
// fixed-point iteration from L = |x_r(t) - x_s(t)|/c (a contraction: |dx_s/dt|/c ~ 1e-4).
bool light_time(const lr_orbit *o, int l, double t, double *out)
{
    int r = LINK_R[l], s = LINK_S[l];
    double xr[3], xs[3];
    for (int d = 0; d < 3; ++d) {
        xr[d] = spline_eval_host(o, 3 * r + d, t);
        xs[d] = spline_eval_host(o, 3 * s + d, t);
    }
    double L = std::sqrt((xr[0] - xs[0]) * (xr[0] - xs[0]) + (xr[1] - xs[1]) * (xr[1] - xs[1]) +
                         (xr[2] - xs[2]) * (xr[2] - xs[2])) / lr::C_LIGHT;
    for (int it = 0; it < 100; ++it) {
        for (int d = 0; d < 3; ++d) xs[d] = spline_eval_host(o, 3 * s + d, t - L);
        double Ln = std::sqrt((xr[0] - xs[0]) * (xr[0] - xs[0]) + (xr[1] - xs[1]) * (xr[1] - xs[1]) +
                              (xr[2] - xs[2]) * (xr[2] - xs[2])) / lr::C_LIGHT;
        double ch = std::fabs(Ln - L);
        L = Ln;
        if (ch <= 1e-15 * L) {
            *out = L;
            return true;
        }
    }
    *out = L;
    return std::isfinite(L);
}

// Inverse of the Vandermonde matrix V_ik = c_i^k of the four Chebyshev nodes
// c_i = cos((2i+1) pi / 8): row k maps node values to the coefficient of s^k of the cubic
// through them (Gauss-Jordan elimination with partial pivoting).
void chebyshev_inverse(double out[4][4], double node[4])
{
    double a[4][8];
    for (int i = 0; i < 4; ++i) {
        double c = std::cos((2.0 * i + 1.0) * 3.14159265358979323846 / 8.0), pw = 1.0;
        node[i] = c;
        for (int k = 0; k < 4; ++k) {
            a[i][k] = pw;
            pw *= c;
            a[i][4 + k] = i == k ? 1.0 : 0.0;
        }
    }
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int r = col + 1; r < 4; ++r)
            if (std::fabs(a[r][col]) > std::fabs(a[piv][col])) piv = r;
        for (int k = 0; k < 8; ++k) std::swap(a[col][k], a[piv][k]);
        double d = a[col][col];
        for (int k = 0; k < 8; ++k) a[col][k] /= d;
        for (int r = 0; r < 4; ++r)
            if (r != col) {
                double f = a[r][col];
                for (int k = 0; k < 8; ++k) a[r][k] -= f * a[col][k];
            }
    }
    // a[:, 4:] = V^{-1}: coefficient k = sum_i V^{-1}[k][i] y_i
    for (int k = 0; k < 4; ++k)
        for (int i = 0; i < 4; ++i) out[k][i] = a[k][4 + i];
}

// Nested chained delays for the mixed kernels (Sec. TDI, the chained delay with each L taken at
// the time the light left: t_k = t_{k-1} - L(t_{k-1})): at every knot t of the TDI orbit and
// for every delayed term (channel, chain, q), the nested total delay minus the summed one
// (all L at t), in samples.  The difference is smooth on orbital time scales (~1e-7 samples,
// second derivative ~1e-20 s/s^2), so the kernels interpolate it linearly per tile.
int nested_table(lr_plan *p, const lr_orbit *o)
{
    const lr::TdiTab tab = lr::make_tdi_tab();
    const int nk = o->nint + 1;
    std::vector<double> h((size_t)nk * 42, 0.0);
    for (int k = 0; k < nk; ++k) {
        const double t = o->t_first + (double)k * o->dk;
        for (int ch = 0; ch < 3; ++ch)
            for (int c = 0; c < 2; ++c) {
                double Dn = 0.0, Ds = 0.0;
                for (int q = 1; q <= 7; ++q) {
                    const int l = tab.pair[ch][c][q];
                    Dn += spline_eval_host(o, 9 + l, t - Dn);
                    Ds += spline_eval_host(o, 9 + l, t);
                    h[(size_t)k * 42 + (ch * 2 + c) * 7 + q - 1] = (Dn - Ds) / p->desc.dt;
                }
            }
    }
    cudaError_t e = lr::dev_malloc((void **)&p->d_nest, sizeof(double) * h.size());
    if (e == cudaSuccess) e = cudaMemcpy(p->d_nest, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (p->d_nest) cudaFree(p->d_nest);
        p->d_nest = nullptr;
        return cuda_fail(p->ctx, e);
    }
    lr::FwdParams &P = p->base;
    P.nest_tab = p->d_nest;
    P.nest_n = nk;
    P.nest_t0 = o->t_first;
    P.nest_inv_dk = 1.0 / o->dk;
    return LR_OK;
}

// Constant TDI delays (Sec. TDI with L_ij independent of t, e.g. the equal-arm template): when
// every delay spline of the TDI orbit is a constant, each chained delay is a constant number of
// samples, so each delayed read has one fractional offset for all outputs.  Its centered Lagrange
// weights (Sec. "Implementation", direct products) and its first tap's offset are computed once
// here; the FP64 kernels then read with a plain dot product.  Nested and summed delays coincide.
int constant_delay_table(lr_plan *p, const lr_orbit *o)
{
    for (int l = 0; l < 6; ++l) {
        const double c0 = o->coef[(size_t)(9 + l) * 4];
        for (int k = 0; k < o->nint; ++k) {
            const double *q = o->coef.data() + ((size_t)k * lr::NSERIES + 9 + l) * 4;
            if (q[0] != c0 || q[1] != 0.0 || q[2] != 0.0 || q[3] != 0.0) return LR_OK;  // not constant
        }
    }
    const int T = p->T, h = p->h;
    const lr::TdiTab tab = lr::make_tdi_tab();
    lr::FwdParams &P = p->base;
    std::vector<double> w((size_t)3 * 2 * lr::CHAIN_TERMS * T, 0.0);
    for (int ch = 0; ch < 3; ++ch)
        for (int c = 0; c < 2; ++c) {
            double D = 0.0;  // samples
            P.cd_off[ch][c][0] = 0;
            for (int q = 1; q < lr::CHAIN_TERMS; ++q) {
                const int l = tab.pair[ch][c][q];
                D += o->coef[(size_t)(9 + l) * 4] * P.inv_dt;
                const double u = -D, fl = std::floor(u), eps = u - fl;
                P.cd_off[ch][c][q] = (int)fl - h;
                double *wq = w.data() + ((size_t)(ch * 2 + c) * lr::CHAIN_TERMS + q) * T;
                for (int a = 0; a < T; ++a) {
                    double prod = 1.0;
                    for (int b = 0; b < T; ++b)
                        if (b != a) prod *= (eps - (double)(b - h)) / (double)(a - b);
                    wq[a] = prod;
                }
            }
        }
    cudaError_t e = lr::dev_malloc((void **)&p->d_cdw, sizeof(double) * w.size());
    if (e == cudaSuccess) e = cudaMemcpy(p->d_cdw, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (p->d_cdw) cudaFree(p->d_cdw);
        p->d_cdw = nullptr;
        return cuda_fail(p->ctx, e);
    }
    P.cd_w = p->d_cdw;
    return LR_OK;
}

bool all_finite(const double *p, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

}  // namespace

// ================================================================== C ABI
extern "C" {

LR_API const char *lr_strerror(int status)
{
    switch (status) {
        case LR_OK: return "success";
        case LR_ERR_INVALID_ARG: return "invalid argument";
        case LR_ERR_RANGE: return "size or value out of the supported range";
        case LR_ERR_OOM: return "out of memory";
        case LR_ERR_CUDA: return "CUDA runtime error";
        case LR_ERR_TIMEOUT: return "bounded device wait ran out";
        case LR_ERR_NONFINITE: return "non-finite input";
        case LR_ERR_UNSUPPORTED: return "unsupported request";
        case LR_ERR_DEVICE: return "kernel recorded an internal fault";
        default: return "unknown status";
    }
}

LR_API int lr_version(void) { return 100; }

LR_API int lr_debug_fail_allocations(int after)
{
    lr::g_alloc_budget = after < 0 ? -1 : after;
    return LR_OK;
}

LR_API int lr_order_supported(int order) { return lr::order_supported(order) ? 1 : 0; }

LR_API int lr_ctx_create(int device, lr_ctx **out)
{
    if (!out || device < 0) return LR_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return LR_ERR_CUDA;
    if (device >= ndev) return LR_ERR_RANGE;
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return LR_ERR_CUDA;
    lr_ctx *c = new (std::nothrow) lr_ctx();
    if (!c) return LR_ERR_OOM;
    c->device = device;
    c->last_cuda_error = 0;
    e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        delete c;
        return LR_ERR_CUDA;
    }
    // the fixed arrays of lr_response_batched_noalloc are resolved (and their module loaded) here
    const int ne = lr::noalloc_setup(device);
    if (ne) {
        c->last_cuda_error = ne;
        delete c;
        return ne == (int)cudaErrorMemoryAllocation ? LR_ERR_OOM : LR_ERR_CUDA;
    }
    *out = c;
    return LR_OK;
}

LR_API int lr_ctx_destroy(lr_ctx *ctx)
{
    if (!ctx) return LR_ERR_INVALID_ARG;
    delete ctx;
    return LR_OK;
}

LR_API int lr_last_cuda_error(const lr_ctx *ctx) { return ctx ? ctx->last_cuda_error : 0; }

LR_API int lr_orbit_create(lr_ctx *ctx, const double *t_knots, int64_t n_knots, const double *pos,
                           const double *delays, int spline_bc, lr_orbit **out)
{
    if (!ctx || !t_knots || !pos || !out) return LR_ERR_INVALID_ARG;
    *out = nullptr;
    if (spline_bc != LR_SPLINE_NOT_A_KNOT && spline_bc != LR_SPLINE_NATURAL) return LR_ERR_INVALID_ARG;
    if (n_knots < 4 || n_knots > (1 << 24)) return LR_ERR_RANGE;
    if (!all_finite(t_knots, (size_t)n_knots) || !all_finite(pos, (size_t)(9 * n_knots))) return LR_ERR_NONFINITE;
    if (delays && !all_finite(delays, (size_t)(6 * n_knots))) return LR_ERR_NONFINITE;
    double dk = (t_knots[n_knots - 1] - t_knots[0]) / (double)(n_knots - 1);
    if (!(dk > 0.0)) return LR_ERR_INVALID_ARG;
    for (int64_t k = 0; k < n_knots; ++k)
        if (std::fabs(t_knots[k] - (t_knots[0] + (double)k * dk)) > 1e-9 * dk) return LR_ERR_INVALID_ARG;

    lr_orbit *o = new (std::nothrow) lr_orbit();
    if (!o) return LR_ERR_OOM;
    o->ctx = ctx;
    o->nk = n_knots;
    o->nint = (int)(n_knots - 1);
    o->t_first = t_knots[0];
    o->dk = dk;
    o->d_coef = nullptr;
    try {
        o->coef.assign((size_t)o->nint * lr::NSERIES * 4, 0.0);
        std::vector<double> M;
        for (int s = 0; s < 9; ++s) {
            if (!spline_second_derivatives(pos + (size_t)s * n_knots, n_knots, dk, spline_bc, M)) {
                delete o;
                return LR_ERR_INVALID_ARG;
            }
            spline_coefficients(pos + (size_t)s * n_knots, M, n_knots, dk, o->coef.data(), s);
        }
        o->delays.assign((size_t)6 * n_knots, 0.0);
        if (delays) {
            std::memcpy(o->delays.data(), delays, sizeof(double) * 6 * (size_t)n_knots);
        } else {
            for (int l = 0; l < 6; ++l)
                for (int64_t k = 0; k < n_knots; ++k)
                    if (!light_time(o, l, t_knots[k], &o->delays[(size_t)l * n_knots + k])) {
                        delete o;
                        return LR_ERR_NONFINITE;
                    }
        }
        for (int l = 0; l < 6; ++l) {
            if (!spline_second_derivatives(o->delays.data() + (size_t)l * n_knots, n_knots, dk, spline_bc, M)) {
                delete o;
                return LR_ERR_INVALID_ARG;
            }
            spline_coefficients(o->delays.data() + (size_t)l * n_knots, M, n_knots, dk, o->coef.data(), 9 + l);
        }
    } catch (const std::bad_alloc &) {
        delete o;
        return LR_ERR_OOM;
    }
    // bounds over the grid, sampled on knots and at 8 points per interval (the cubic pieces
    // of smooth orbits overshoot their knot values only by a tiny amount)
    double rmax = 0.0, lmax = 0.0, vmax = 0.0, ldot = 0.0;
    for (int k = 0; k < o->nint; ++k)
        for (int j = 0; j <= 8; ++j) {
            double t = o->t_first + ((double)k + j / 8.0) * dk;
            // derivative of each cubic piece: (b + 2 c x + 3 d x^2) / dk
            const double x = j / 8.0;
            for (int s = 0; s < lr::NSERIES; ++s) {
                const double *q = o->coef.data() + ((size_t)k * lr::NSERIES + s) * 4;
                double dv = std::fabs((q[1] + x * (2.0 * q[2] + 3.0 * x * q[3])) / dk);
                if (s < 9) vmax = std::max(vmax, dv); else ldot = std::max(ldot, dv);
            }
            for (int i = 0; i < 3; ++i) {
                double r2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                    double v = spline_eval_host(o, 3 * i + d, t);
                    r2 += v * v;
                }
                rmax = std::max(rmax, std::sqrt(r2));
            }
            for (int l = 0; l < 6; ++l) lmax = std::max(lmax, std::fabs(spline_eval_host(o, 9 + l, t)));
        }
    o->max_r_over_c = rmax / lr::C_LIGHT * (1.0 + 1e-3) + 1e-3;
    o->max_delay = lmax * (1.0 + 1e-3) + 1e-3;
    o->max_rate = (std::sqrt(3.0) * vmax / lr::C_LIGHT + ldot) * 1.1 + 1e-9;
    for (size_t i = 0; i < o->delays.size(); ++i)
        if (!(o->delays[i] > 0.0)) {
            delete o;
            return LR_ERR_RANGE;  // light travel times are positive
        }
    cudaError_t e = lr::dev_malloc((void **)&o->d_coef, sizeof(double) * o->coef.size());
    if (e != cudaSuccess) {
        delete o;
        return e == cudaErrorMemoryAllocation ? LR_ERR_OOM : cuda_fail(ctx, e);
    }
    e = cudaMemcpy(o->d_coef, o->coef.data(), sizeof(double) * o->coef.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(o->d_coef);
        delete o;
        return cuda_fail(ctx, e);
    }
    *out = o;
    return LR_OK;
}

LR_API int lr_orbit_destroy(lr_orbit *orbit)
{
    if (!orbit) return LR_ERR_INVALID_ARG;
    if (orbit->d_coef) cudaFree(orbit->d_coef);
    delete orbit;
    return LR_OK;
}

LR_API int lr_orbit_delays(const lr_orbit *orbit, double *out, int64_t n_knots)
{
    if (!orbit || !out) return LR_ERR_INVALID_ARG;
    if (n_knots != orbit->nk) return LR_ERR_RANGE;
    std::memcpy(out, orbit->delays.data(), sizeof(double) * orbit->delays.size());
    return LR_OK;
}

LR_API int lr_plan_create(lr_ctx *ctx, const lr_plan_desc *d, lr_plan **out)
{
    if (!ctx || !d || !out) return LR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!d->proj_orbit || !d->tdi_orbit) return LR_ERR_INVALID_ARG;
    if (d->order < 1 || d->order > 63) return LR_ERR_RANGE;
    if ((d->order & 1) == 0) return LR_ERR_UNSUPPORTED;
    if (!lr::order_supported(d->order)) return LR_ERR_UNSUPPORTED;
    if (d->precision != LR_FP64 && d->precision != LR_MIXED) return LR_ERR_INVALID_ARG;
    if (d->tdi_generation != 1 && d->tdi_generation != 2) return LR_ERR_INVALID_ARG;
    if (d->delay_mode != LR_DELAY_SUM && d->delay_mode != LR_DELAY_NESTED) return LR_ERR_INVALID_ARG;
    if (!(d->dt > 0.0) || !std::isfinite(d->dt) || !std::isfinite(d->t0)) return LR_ERR_INVALID_ARG;
    if (d->n < 1) return LR_ERR_INVALID_ARG;
    if (d->tile < 0 || d->tile > 8192 || d->threads < 0 || d->threads > 1024) return LR_ERR_RANGE;
    if (d->threads && (d->threads % 32)) return LR_ERR_INVALID_ARG;
    if (!lr::precision_supported(d->precision)) return LR_ERR_UNSUPPORTED;

    lr_plan *p = new (std::nothrow) lr_plan();
    if (!p) return LR_ERR_OOM;
    p->ctx = ctx;
    p->desc = *d;
    p->T = d->order + 1;
    p->h = (d->order - 1) / 2;
    p->threads = d->threads ? d->threads : 256;
    p->d_err = nullptr;
    p->d_tile_off = nullptr;
    p->tile_cap = 0;
    p->d_gy = nullptr;
    p->gy_cap = 0;
    p->d_partial = nullptr;
    p->partial_cap = 0;
    p->d_ktile_off = p->d_htile_off = nullptr;
    p->ktile_cap = 0;
    p->pipe = nullptr;
    p->d_lpart = nullptr;
    p->lpart_cap = 0;
    p->d_nest = nullptr;
    p->d_cdw = nullptr;
    lr::FwdParams &P = p->base;
    std::memset(&P, 0, sizeof(P));
    P.dt = d->dt;
    P.inv_dt = 1.0 / d->dt;
    P.t0 = d->t0;
    P.po = {d->proj_orbit->d_coef, d->proj_orbit->nint, d->proj_orbit->t_first, 1.0 / d->proj_orbit->dk};
    P.to = {d->tdi_orbit->d_coef, d->tdi_orbit->nint, d->tdi_orbit->t_first, 1.0 / d->tdi_orbit->dk};
    P.q_terms = d->tdi_generation == 1 ? 3 : 7;
    P.delay_nested = d->delay_mode == LR_DELAY_NESTED;
    P.tile = d->tile;
    // a chained delay is at most q_terms link delays; a tile's link series extend by that
    // plus the stencil on the left and by the stencil on the right
    double chain = (double)P.q_terms * d->tdi_orbit->max_delay / d->dt;
    if (chain > 1e6) {
        delete p;
        return LR_ERR_RANGE;
    }
    P.HL = (int)std::ceil(chain) + p->h + 2;
    P.HR = p->h + 2;
    double sig = d->proj_orbit->max_r_over_c / d->dt;
    double lp = d->proj_orbit->max_delay / d->dt;
    if (sig > 1e6 || lp > 1e6) {
        delete p;
        return LR_ERR_RANGE;
    }
    P.sig_b = (int)std::ceil(sig) + 1;
    P.lproj_b = (int)std::ceil(lp) + 1;
    if (d->precision == LR_MIXED) {
        // mixed tiles are staged in fixed shared-memory arrays: the largest tile that fits
        const int tmax = lr::mx_max_tile(P.HL, P.HR, P.lproj_b, p->T);
        if (tmax < 4 || (P.tile != 0 && P.tile > tmax)) {
            delete p;
            return LR_ERR_RANGE;
        }
        if (P.tile == 0) P.tile = tmax;
    } else if (P.tile == 0) {
        P.tile = lr::default_tile(d->precision, d->order);
    }
    P.ymax = P.tile + P.HL + P.HR;
    P.wmax = P.ymax + 2 * P.sig_b + P.lproj_b + p->T + 4;
    if (d->precision == LR_MIXED) {
        // the mixed kernels re-expand the orbit cubics over a tile: a tile's link span must fit
        // in two knot intervals
        if ((double)P.ymax * d->dt >= d->proj_orbit->dk || (double)P.tile * d->dt >= d->tdi_orbit->dk) {
            delete p;
            return LR_ERR_RANGE;
        }
    }
    chebyshev_inverse(P.cheb, P.cheb_node);
    cudaError_t e = lr::dev_malloc((void **)&p->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        if (p->d_err) cudaFree(p->d_err);
        delete p;
        return cuda_fail(ctx, e);
    }
    P.err = p->d_err;
    if (d->precision == LR_MIXED && d->delay_mode == LR_DELAY_NESTED) {
        const int st = nested_table(p, d->tdi_orbit);
        if (st) {
            cudaFree(p->d_err);
            delete p;
            return st;
        }
    }
    if (d->precision == LR_FP64) {
        const int st = constant_delay_table(p, d->tdi_orbit);
        if (st) {
            cudaFree(p->d_err);
            delete p;
            return st;
        }
    }
    *out = p;
    return LR_OK;
}

LR_API int lr_plan_destroy(lr_plan *plan)
{
    if (!plan) return LR_ERR_INVALID_ARG;
    if (plan->d_err) cudaFree(plan->d_err);
    if (plan->d_tile_off) cudaFree(plan->d_tile_off);
    if (plan->d_gy) cudaFree(plan->d_gy);
    if (plan->d_partial) cudaFree(plan->d_partial);
    if (plan->d_ktile_off) cudaFree(plan->d_ktile_off);
    if (plan->d_htile_off) cudaFree(plan->d_htile_off);
    if (plan->d_lpart) cudaFree(plan->d_lpart);
    if (plan->d_nest) cudaFree(plan->d_nest);
    if (plan->d_cdw) cudaFree(plan->d_cdw);
    lr::pipe_free(plan->pipe);
    delete plan;
    return LR_OK;
}

LR_API int lr_required_margin(const lr_plan *plan, int64_t *left, int64_t *right)
{
    if (!plan || !left || !right) return LR_ERR_INVALID_ARG;
    *left = plan->base.sig_b + plan->base.lproj_b + plan->h + 2;
    *right = plan->base.sig_b + plan->h + 2;
    return LR_OK;
}

LR_API int lr_plan_tile(const lr_plan *plan, int *tile)
{
    if (!plan || !tile) return LR_ERR_INVALID_ARG;
    *tile = plan->base.tile;
    return LR_OK;
}

LR_API int lr_valid_range(const lr_plan *plan, int64_t *first, int64_t *last)
{
    if (!plan || !first || !last) return LR_ERR_INVALID_ARG;
    // the chained delays reach back by at most q_terms link delays; a read at fractional
    // position x uses samples floor(x) - h .. floor(x) + h + 1
    const double chain = (double)plan->base.q_terms * plan->desc.tdi_orbit->max_delay / plan->desc.dt;
    *first = (int64_t)std::ceil(chain) + plan->h + 1;
    *last = plan->desc.n - 2 - plan->h;
    return LR_OK;
}

LR_API int lr_plan_check(lr_plan *plan, void *stream)
{
    if (!plan) return LR_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(plan->ctx, e);
    int flag = 0;
    e = cudaMemcpy(&flag, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(plan->ctx, e);
    if (flag) {
        e = cudaMemset(plan->d_err, 0, sizeof(int));
        if (e != cudaSuccess) return cuda_fail(plan->ctx, e);
    }
    if (flag & lr::ERR_TIMEOUT) return LR_ERR_TIMEOUT;
    if (flag == lr::ERR_NONFINITE) return LR_ERR_NONFINITE;
    if (flag) return LR_ERR_DEVICE;
    return LR_OK;
}

}  // extern "C"

namespace {

// Sizes the backward launch parameters and grows the plan's workspace.
int backward_setup(lr_plan *plan, int64_t gy_elems, int64_t ktiles, lr::FwdParams &P, lr::BwdParams &B)
{
    P = plan->base;
    std::memset(&B, 0, sizeof(B));
    P.tile = lr::BWD_TILE_K;
    P.wmax = lr::BWD_TILE_K + 2 * P.sig_b + P.lproj_b + plan->T + 4;
    const double chain = (double)P.q_terms * plan->desc.tdi_orbit->max_delay / plan->desc.dt;
    B.dmax = (int)std::ceil(chain) + 1;
    B.tile_h = lr::BWD_TILE_H;
    B.wn = lr::BWD_TILE_K + 2 * plan->h + 5 + B.dmax;
    const double span = (double)(lr::BWD_TILE_H + plan->T + 2 * (P.sig_b + P.lproj_b));
    B.kmargin = 2 + (int)std::ceil(plan->desc.proj_orbit->max_rate * span);
    B.wk = lr::BWD_TILE_H + plan->T + 5 + 2 * P.lproj_b + 2 * B.kmargin;
    if (gy_elems > plan->gy_cap) {
        if (plan->d_gy) cudaFree(plan->d_gy);
        plan->d_gy = nullptr;
        plan->gy_cap = 0;
        cudaError_t e = lr::dev_malloc((void **)&plan->d_gy, sizeof(double) * (size_t)gy_elems);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LR_ERR_OOM : cuda_fail(plan->ctx, e);
        plan->gy_cap = gy_elems;
    }
    if (3 * ktiles > plan->partial_cap) {
        if (plan->d_partial) cudaFree(plan->d_partial);
        plan->d_partial = nullptr;
        plan->partial_cap = 0;
        cudaError_t e = lr::dev_malloc((void **)&plan->d_partial, sizeof(double) * (size_t)(3 * ktiles));
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LR_ERR_OOM : cuda_fail(plan->ctx, e);
        plan->partial_cap = 3 * ktiles;
    }
    B.g_y = plan->d_gy;
    B.partial = plan->d_partial;
    return LR_OK;
}

// TDI transpose, sky partials, projection transpose, then the ordered sky reduction.
int backward_launch(lr_plan *plan, lr::FwdParams &P, lr::BwdParams &B, int64_t S, const int64_t *ktile_off,
                    double *g_sky, void *stream)
{
    const int sms = plan->ctx->sms;
    const int order = plan->desc.order;
    // mixed plans: the transposes and the sky gradient in the mixed kernels
    const bool mx = plan->desc.precision == LR_MIXED;
    int e = mx ? lr::launch_bwd_mx(0, order, P, B, sms, stream) : lr::launch_bwd(0, order, P, B, sms, stream);
    if (!e && g_sky) e = mx ? lr::launch_bwd_mx(2, order, P, B, sms, stream) : lr::launch_bwd(2, order, P, B, sms, stream);
    if (!e) e = mx ? lr::launch_bwd_mx(1, order, P, B, sms, stream) : lr::launch_bwd(1, order, P, B, sms, stream);
    if (!e && g_sky) e = lr::launch_sky_reduce(B.partial, ktile_off, S, P.total_tiles, g_sky, stream);
    return check_launch(plan->ctx, e);
}

}  // namespace

// ================================================================== launches
namespace {

int launch_single(lr_plan *plan, int kind, lr::FwdParams &P, void *stream)
{
    const int64_t n = plan->desc.n;
    P.total_tiles = (n + P.tile - 1) / P.tile;
    return check_launch(plan->ctx, lr::launch_forward(plan->desc.precision, kind, plan->desc.order, P,
                                                      plan->threads, plan->ctx->sms, stream));
}

}  // namespace

extern "C" {

LR_API int lr_project(lr_plan *plan, const double *hp, const double *hc, int64_t n_h, double t0_h, lr_sky sky,
                      double *y, void *stream)
{
    if (!plan || !hp || !hc || !y) return LR_ERR_INVALID_ARG;
    if (n_h < 1) return LR_ERR_INVALID_ARG;
    if (!std::isfinite(t0_h) || !std::isfinite(sky.lam) || !std::isfinite(sky.beta) || !std::isfinite(sky.psi))
        return LR_ERR_NONFINITE;
    if (std::fabs(plan->desc.t0 - t0_h) / plan->desc.dt > 1e12) return LR_ERR_RANGE;
    lr::FwdParams P = plan->base;
    P.src.n1 = plan->desc.n;
    P.src.nh1 = n_h;
    P.src.t0h1 = t0_h;
    P.src.sky1 = sky;
    P.src.skyc1 = lr::make_sky(sky);
    P.hp = hp;
    P.hc = hc;
    P.out = y;
    return launch_single(plan, lr::KIND_PROJECT, P, stream);
}

LR_API int lr_tdi(lr_plan *plan, const double *y, double *xyz, void *stream)
{
    if (!plan || !y || !xyz) return LR_ERR_INVALID_ARG;
    lr::FwdParams P = plan->base;
    P.src.n1 = plan->desc.n;
    P.src.nh1 = 0;
    P.yin = y;
    P.out = xyz;
    return launch_single(plan, lr::KIND_TDI, P, stream);
}

LR_API int lr_response(lr_plan *plan, const double *hp, const double *hc, int64_t n_h, double t0_h, lr_sky sky,
                       double *xyz, void *stream)
{
    if (!plan || !hp || !hc || !xyz) return LR_ERR_INVALID_ARG;
    if (n_h < 1) return LR_ERR_INVALID_ARG;
    if (!std::isfinite(t0_h) || !std::isfinite(sky.lam) || !std::isfinite(sky.beta) || !std::isfinite(sky.psi))
        return LR_ERR_NONFINITE;
    if (std::fabs(plan->desc.t0 - t0_h) / plan->desc.dt > 1e12) return LR_ERR_RANGE;
    lr::FwdParams P = plan->base;
    P.src.n1 = plan->desc.n;
    P.src.nh1 = n_h;
    P.src.t0h1 = t0_h;
    P.src.sky1 = sky;
    P.src.skyc1 = lr::make_sky(sky);
    P.hp = hp;
    P.hc = hc;
    P.out = xyz;
    return launch_single(plan, lr::KIND_FUSED, P, stream);
}

}  // extern "C"

namespace {

// the batched fused launch; gb != null: Galactic binaries generated on the device (h_off, t0_h,
// hp, hc unused)
int response_batched_impl(lr_plan *plan, int64_t S, const int64_t *h_off, const int64_t *out_off, const double *t0_h,
                          const lr_sky *sky, const double *hp, const double *hc, const lr_gb *gb, double *xyz,
                          void *stream)
{
    if (!plan || !out_off || !sky || !xyz) return LR_ERR_INVALID_ARG;
    if (!gb && (!h_off || !t0_h || !hp || !hc)) return LR_ERR_INVALID_ARG;
    if (S < 1) return LR_ERR_INVALID_ARG;
    if (S > (int64_t)1 << 24) return LR_ERR_RANGE;
    int st = lr::plan_reserve_batch(plan, S);
    if (st) return st;
    lr::FwdParams P = plan->base;
    lr::SkyConst *skyc = plan->desc.precision == LR_MIXED ? lr::plan_sky_table(plan) : nullptr;
    int e = lr::launch_batch_tables(out_off, sky, S, P.tile, plan->d_tile_off, skyc, P.err, stream);
    if (e) return check_launch(plan->ctx, e);
    P.src.skyc = skyc;
    P.src.h_off = h_off;
    P.src.out_off = out_off;
    P.src.t0h = t0_h;
    P.src.sky = sky;
    P.src.tile_off = plan->d_tile_off;
    P.src.S = S;
    P.src.gb = gb;
    P.gen_strain = gb != nullptr;
    P.hp = hp;
    P.hc = hc;
    P.out = xyz;
    P.total_tiles = -1;
    return check_launch(plan->ctx, lr::launch_forward(plan->desc.precision, lr::KIND_FUSED, plan->desc.order, P,
                                                      plan->threads, plan->ctx->sms, stream));
}

bool gb_finite(const lr_gb &g)
{
    return std::isfinite(g.A) && std::isfinite(g.f0) && std::isfinite(g.fdot) && std::isfinite(g.fddot) &&
           std::isfinite(g.phi0) && std::isfinite(g.iota);
}

}  // namespace

extern "C" {

LR_API int lr_response_batched(lr_plan *plan, int64_t S, const int64_t *h_off, const int64_t *out_off,
                               const double *t0_h, const lr_sky *sky, const double *hp, const double *hc,
                               double *xyz, void *stream)
{
    if (!h_off || !t0_h || !hp || !hc) return LR_ERR_INVALID_ARG;
    return response_batched_impl(plan, S, h_off, out_off, t0_h, sky, hp, hc, nullptr, xyz, stream);
}

LR_API int lr_response_gb_batched(lr_plan *plan, int64_t S, const int64_t *out_off, const lr_gb *gb,
                                  const lr_sky *sky, double *xyz, void *stream)
{
    if (!gb) return LR_ERR_INVALID_ARG;
    return response_batched_impl(plan, S, nullptr, out_off, nullptr, sky, nullptr, nullptr, gb, xyz, stream);
}

LR_API int lr_response_gb(lr_plan *plan, lr_gb gb, lr_sky sky, double *xyz, void *stream)
{
    if (!plan || !xyz) return LR_ERR_INVALID_ARG;
    if (!gb_finite(gb) || !std::isfinite(sky.lam) || !std::isfinite(sky.beta) || !std::isfinite(sky.psi))
        return LR_ERR_NONFINITE;
    lr::FwdParams P = plan->base;
    P.src.n1 = plan->desc.n;
    P.src.nh1 = lr::GEN_STRAIN_LEN;
    P.src.t0h1 = plan->desc.t0;
    P.src.sky1 = sky;
    P.src.skyc1 = lr::make_sky(sky);
    P.src.gb1 = gb;
    P.gen_strain = 1;
    P.out = xyz;
    return launch_single(plan, lr::KIND_FUSED, P, stream);
}

}  // extern "C"

namespace {

// validates the weights and sizes the per-tile partial buffer for `tiles` tiles
int like_setup(lr_plan *plan, const double *weights, int64_t tiles, lr::FwdParams &P, const double *data,
               int64_t n_total)
{
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(weights[c]) || weights[c] < 0.0) return LR_ERR_INVALID_ARG;
    if (tiles > plan->lpart_cap) {
        if (plan->d_lpart) cudaFree(plan->d_lpart);
        plan->d_lpart = nullptr;
        plan->lpart_cap = 0;
        cudaError_t e = lr::dev_malloc((void **)&plan->d_lpart, sizeof(double) * 2 * (size_t)tiles);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LR_ERR_OOM : cuda_fail(plan->ctx, e);
        plan->lpart_cap = tiles;
    }
    P.like.data = data;
    double wmax = 0.0;
    for (int c = 0; c < 3; ++c) {
        P.like.w[c] = weights[c];
        wmax = std::max(wmax, weights[c]);
    }
    P.like.wmax = wmax;
    for (int c = 0; c < 3; ++c) P.like.wn[c] = wmax > 0.0 ? (float)(weights[c] / wmax) : 0.0f;
    P.like.partial = plan->d_lpart;
    P.like.cap = plan->lpart_cap;
    P.like.n_total = n_total;
    return LR_OK;
}

// the mixed epilogue sums with the weights normalised to the largest one
double like_post(const lr_plan *plan, const lr::FwdParams &P)
{
    return plan->desc.precision == LR_MIXED ? P.like.wmax : 1.0;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// the fused likelihood launch and its per-source reduction; logl selects the output form
int likelihood_single(lr_plan *plan, const double *hp, const double *hc, int64_t n_h, double t0_h, lr_sky sky,
                      const double *data, const double *weights, int logl, double *dh_hh, double *xyz, void *stream)
{
    if (!plan || !hp || !hc || !data || !weights || !dh_hh) return LR_ERR_INVALID_ARG;
    if (n_h < 1) return LR_ERR_INVALID_ARG;
    if (!std::isfinite(t0_h) || !std::isfinite(sky.lam) || !std::isfinite(sky.beta) || !std::isfinite(sky.psi))
        return LR_ERR_NONFINITE;
    if (std::fabs(plan->desc.t0 - t0_h) / plan->desc.dt > 1e12) return LR_ERR_RANGE;
    lr::FwdParams P = plan->base;
    const int64_t n = plan->desc.n, tiles = (n + P.tile - 1) / P.tile;
    int st = like_setup(plan, weights, tiles, P, data, n);
    if (st) return st;
    P.src.n1 = n;
    P.src.nh1 = n_h;
    P.src.t0h1 = t0_h;
    P.src.sky1 = sky;
    P.src.skyc1 = lr::make_sky(sky);
    P.hp = hp;
    P.hc = hc;
    P.out = xyz;
    st = launch_single(plan, lr::KIND_LIKE, P, stream);
    if (st) return st;
    return check_launch(plan->ctx, lr::launch_like_reduce(plan->d_lpart, nullptr, tiles, 1, plan->lpart_cap,
                                                          like_post(plan, P), logl, dh_hh, plan->d_err, stream));
}

int likelihood_batched(lr_plan *plan, int64_t S, const int64_t *h_off, const int64_t *out_off, const double *t0_h,
                       const lr_sky *sky, const double *hp, const double *hc, const lr_gb *gb, const double *data,
                       int64_t n_total, const double *weights, int logl, double *dh_hh, double *xyz, void *stream)
{
    if (!plan || !out_off || !sky || !data || !weights || !dh_hh) return LR_ERR_INVALID_ARG;
    if (!gb && (!h_off || !t0_h || !hp || !hc)) return LR_ERR_INVALID_ARG;
    if (S < 1 || n_total < 0) return LR_ERR_INVALID_ARG;
    if (S > (int64_t)1 << 24 || n_total > (int64_t)1 << 40) return LR_ERR_RANGE;
    int st = lr::plan_reserve_batch(plan, S);
    if (st) return st;
    lr::FwdParams P = plan->base;
    // sum over sources of ceil(N_s / tile) <= n_total / tile + S
    st = like_setup(plan, weights, n_total / P.tile + S, P, data, n_total);
    if (st) return st;
    lr::SkyConst *skyc = plan->desc.precision == LR_MIXED ? lr::plan_sky_table(plan) : nullptr;
    int e = lr::launch_batch_tables(out_off, sky, S, P.tile, plan->d_tile_off, skyc, P.err, stream);
    if (e) return check_launch(plan->ctx, e);
    P.src.skyc = skyc;
    P.src.h_off = h_off;
    P.src.out_off = out_off;
    P.src.t0h = t0_h;
    P.src.sky = sky;
    P.src.tile_off = plan->d_tile_off;
    P.src.S = S;
    P.src.gb = gb;
    P.gen_strain = gb != nullptr;
    P.hp = hp;
    P.hc = hc;
    P.out = xyz;
    P.total_tiles = -1;
    st = check_launch(plan->ctx, lr::launch_forward(plan->desc.precision, lr::KIND_LIKE, plan->desc.order, P,
                                                    plan->threads, plan->ctx->sms, stream));
    if (st) return st;
    return check_launch(plan->ctx, lr::launch_like_reduce(plan->d_lpart, plan->d_tile_off, 0, S, plan->lpart_cap,
                                                          like_post(plan, P), logl, dh_hh, plan->d_err, stream));
}

}  // namespace

extern "C" {

LR_API int lr_likelihood(lr_plan *plan, const double *hp, const double *hc, int64_t n_h, double t0_h, lr_sky sky,
                         const double *data, const double *weights, double *dh_hh, double *xyz, void *stream)
{
    return likelihood_single(plan, hp, hc, n_h, t0_h, sky, data, weights, 0, dh_hh, xyz, stream);
}

LR_API int lr_likelihood_batched(lr_plan *plan, int64_t S, const int64_t *h_off, const int64_t *out_off,
                                 const double *t0_h, const lr_sky *sky, const double *hp, const double *hc,
                                 const double *data, int64_t n_total, const double *weights, double *dh_hh,
                                 double *xyz, void *stream)
{
    if (!h_off || !t0_h || !hp || !hc) return LR_ERR_INVALID_ARG;
    return likelihood_batched(plan, S, h_off, out_off, t0_h, sky, hp, hc, nullptr, data, n_total, weights, 0, dh_hh,
                              xyz, stream);
}

LR_API int lr_log_likelihood(lr_plan *plan, const double *hp, const double *hc, int64_t n_h, double t0_h,
                             lr_sky sky, const double *data, const double *weights, double *logl, double *xyz,
                             void *stream)
{
    return likelihood_single(plan, hp, hc, n_h, t0_h, sky, data, weights, 1, logl, xyz, stream);
}

LR_API int lr_log_likelihood_batched(lr_plan *plan, int64_t S, const int64_t *h_off, const int64_t *out_off,
                                     const double *t0_h, const lr_sky *sky, const double *hp, const double *hc,
                                     const double *data, int64_t n_total, const double *weights, double *logl,
                                     double *xyz, void *stream)
{
    if (!h_off || !t0_h || !hp || !hc) return LR_ERR_INVALID_ARG;
    return likelihood_batched(plan, S, h_off, out_off, t0_h, sky, hp, hc, nullptr, data, n_total, weights, 1, logl,
                              xyz, stream);
}

LR_API int lr_log_likelihood_gb_batched(lr_plan *plan, int64_t S, const int64_t *out_off, const lr_gb *gb,
                                        const lr_sky *sky, const double *data, int64_t n_total, const double *weights,
                                        double *logl, double *xyz, void *stream)
{
    if (!gb) return LR_ERR_INVALID_ARG;
    return likelihood_batched(plan, S, nullptr, out_off, nullptr, sky, nullptr, nullptr, gb, data, n_total, weights, 1,
                              logl, xyz, stream);
}

LR_API int lr_likelihood_grad(lr_plan *plan, const double *xyz, const double *data, const double *weights,
                              double scale, double *g_xyz, void *stream)
{
    if (!plan) return LR_ERR_INVALID_ARG;
    return lr_likelihood_grad_batched(plan, 1, nullptr, plan->desc.n, xyz, data, weights, scale, g_xyz, stream);
}

LR_API int lr_likelihood_grad_batched(lr_plan *plan, int64_t S, const int64_t *out_off, int64_t n_total,
                                      const double *xyz, const double *data, const double *weights, double scale,
                                      double *g_xyz, void *stream)
{
    if (!plan || !xyz || !data || !weights || !g_xyz) return LR_ERR_INVALID_ARG;
    if (S < 1 || n_total < 0 || (!out_off && S != 1)) return LR_ERR_INVALID_ARG;
    if (S > (int64_t)1 << 24) return LR_ERR_RANGE;
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(weights[c]) || weights[c] < 0.0) return LR_ERR_INVALID_ARG;
    if (!std::isfinite(scale)) return LR_ERR_NONFINITE;
    return check_launch(plan->ctx, lr::launch_like_grad(out_off, S, n_total, xyz, data, weights, scale, g_xyz,
                                                        plan->d_err, stream));
}

LR_API int lr_backward(lr_plan *plan, const double *hp, const double *hc, int64_t n_h, double t0_h, lr_sky sky,
                       const double *g_xyz, double *g_hp, double *g_hc, double *g_sky, void *stream)
{
    if (!plan || !hp || !hc || !g_xyz || !g_hp || !g_hc) return LR_ERR_INVALID_ARG;
    if (n_h < 1) return LR_ERR_INVALID_ARG;
    if (!std::isfinite(t0_h) || !std::isfinite(sky.lam) || !std::isfinite(sky.beta) || !std::isfinite(sky.psi))
        return LR_ERR_NONFINITE;
    if (std::fabs(plan->desc.t0 - t0_h) / plan->desc.dt > 1e12) return LR_ERR_RANGE;
    lr::FwdParams P;
    lr::BwdParams B;
    const int64_t N = plan->desc.n;
    const int64_t ktiles = (N + lr::BWD_TILE_K - 1) / lr::BWD_TILE_K;
    int st = backward_setup(plan, 6 * N, ktiles, P, B);
    if (st) return st;
    P.src.n1 = N;
    P.src.nh1 = n_h;
    P.src.t0h1 = t0_h;
    P.src.sky1 = sky;
    P.hp = hp;
    P.hc = hc;
    P.out = const_cast<double *>(g_xyz);  // base of the per-source output offsets
    P.total_tiles = ktiles;
    B.g_xyz = g_xyz;
    B.g_hp = g_hp;
    B.g_hc = g_hc;
    B.h_tile_off = nullptr;
    B.h_total_tiles = (n_h + lr::BWD_TILE_H - 1) / lr::BWD_TILE_H;
    return backward_launch(plan, P, B, 1, nullptr, g_sky, stream);
}

LR_API int lr_backward_batched(lr_plan *plan, int64_t S, const int64_t *h_off, const int64_t *out_off,
                               const double *t0_h, const lr_sky *sky, const double *hp, const double *hc,
                               const double *g_xyz, double *g_hp, double *g_hc, double *g_sky, void *stream)
{
    if (!plan || !h_off || !out_off || !t0_h || !sky || !hp || !hc || !g_xyz || !g_hp || !g_hc)
        return LR_ERR_INVALID_ARG;
    if (S < 1) return LR_ERR_INVALID_ARG;
    if (S > (int64_t)1 << 24) return LR_ERR_RANGE;
    // the workspace is sized from the total output length: one small device-to-host read
    int64_t total_n = 0;
    cudaError_t e = cudaMemcpyAsync(&total_n, out_off + S, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                    (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(plan->ctx, e);
    if (total_n < 0) return LR_ERR_INVALID_ARG;
    const int64_t ktiles_bound = total_n / lr::BWD_TILE_K + S + 1;
    lr::FwdParams P;
    lr::BwdParams B;
    int st = backward_setup(plan, 6 * (total_n > 0 ? total_n : 1), ktiles_bound, P, B);
    if (st) return st;
    if (S + 1 > plan->ktile_cap) {
        if (plan->d_ktile_off) cudaFree(plan->d_ktile_off);
        if (plan->d_htile_off) cudaFree(plan->d_htile_off);
        plan->d_ktile_off = plan->d_htile_off = nullptr;
        plan->ktile_cap = 0;
        e = lr::dev_malloc((void **)&plan->d_ktile_off, sizeof(int64_t) * (size_t)(S + 1));
        if (e == cudaSuccess) e = lr::dev_malloc((void **)&plan->d_htile_off, sizeof(int64_t) * (size_t)(S + 1));
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LR_ERR_OOM : cuda_fail(plan->ctx, e);
        plan->ktile_cap = S + 1;
    }
    int le = lr::launch_tile_offsets(out_off, S, lr::BWD_TILE_K, plan->d_ktile_off, P.err, stream);
    if (!le) le = lr::launch_tile_offsets(h_off, S, lr::BWD_TILE_H, plan->d_htile_off, P.err, stream);
    if (le) return check_launch(plan->ctx, le);
    P.src.h_off = h_off;
    P.src.out_off = out_off;
    P.src.t0h = t0_h;
    P.src.sky = sky;
    P.src.tile_off = plan->d_ktile_off;
    P.src.S = S;
    P.hp = hp;
    P.hc = hc;
    P.out = const_cast<double *>(g_xyz);
    P.total_tiles = -1;
    B.g_xyz = g_xyz;
    B.g_hp = g_hp;
    B.g_hc = g_hc;
    B.h_tile_off = plan->d_htile_off;
    B.h_total_tiles = -1;
    return backward_launch(plan, P, B, S, plan->d_ktile_off, g_sky, stream);
}

}  // extern "C"

// ================================================================== plan view
namespace lr {

int plan_view(const lr_plan *plan, PlanView *v)
{
    if (!plan || !v) return LR_ERR_INVALID_ARG;
    v->base = plan->base;
    v->precision = plan->desc.precision;
    v->order = plan->desc.order;
    v->threads = plan->threads;
    v->sms = plan->ctx->sms;
    v->device = plan->ctx->device;
    return LR_OK;
}

int plan_cuda_fail(lr_plan *plan, int cuda_error) { return cuda_fail(plan ? plan->ctx : nullptr, (cudaError_t)cuda_error); }

int plan_set_tile(lr_plan *plan, int tile)
{
    if (!plan) return LR_ERR_INVALID_ARG;
    if (tile < 16 || tile > 8192) return LR_ERR_RANGE;
    FwdParams &P = plan->base;
    const int ymax = tile + P.HL + P.HR;
    if (plan->desc.precision == LR_MIXED &&
        ((double)ymax * plan->desc.dt >= plan->desc.proj_orbit->dk || (double)tile * plan->desc.dt >= plan->desc.tdi_orbit->dk ||
         tile > lr::mx_max_tile(P.HL, P.HR, P.lproj_b, plan->T)))
        return LR_ERR_RANGE;
    P.tile = tile;
    P.ymax = ymax;
    P.wmax = P.ymax + 2 * P.sig_b + P.lproj_b + plan->T + 4;
    return LR_OK;
}

int plan_reserve_batch(lr_plan *plan, int64_t S)
{
    if (!plan) return LR_ERR_INVALID_ARG;
    if (S + 1 <= plan->tile_cap) return LR_OK;
    if (plan->d_tile_off) cudaFree(plan->d_tile_off);
    plan->d_tile_off = nullptr;
    plan->tile_cap = 0;
    // one allocation: the tile table [S+1] followed by the sky frames [S+1]
    const size_t bytes = (sizeof(int64_t) + sizeof(SkyConst)) * (size_t)(S + 1);
    cudaError_t e = lr::dev_malloc((void **)&plan->d_tile_off, bytes);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LR_ERR_OOM : cuda_fail(plan->ctx, e);
    plan->tile_cap = S + 1;
    return LR_OK;
}

PipeWork *&plan_pipe(lr_plan *plan) { return plan->pipe; }

SkyConst *plan_sky_table(lr_plan *plan) { return reinterpret_cast<SkyConst *>(plan->d_tile_off + plan->tile_cap); }

}  // namespace lr
