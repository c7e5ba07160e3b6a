// Mixed-precision forward kernels (FP32 taps and accumulation of the interpolated strain,
// float-float link series and TDI sums, FP64 for times, spline and delay evaluation).
//
// Per tile of output samples a CTA
//  1. builds, in FP64, the cubic of every read position (3 reception reads, 6 emission reads)
//     and of every TDI delay over the tile's knot interval(s) - exact re-expansions of the orbit
//     splines - and fits the 12 smooth geometry factors den_l * xi_l over the tile;
//  2. stages the strain window scaled by a power of two (so FP32 never underflows), as
//     float-float values and first differences plus second and third differences;
//  3. computes the six link series of the tile and its TDI halo in float-float (compensated
//     reads, see lr_mixed.cuh) and stages them the same way;
//  4. forms X, Y, Z: per sample the chained delays are exact 64-bit fixed-point sums of the
//     FP64-evaluated delays, split exactly into index and fraction; the FP32 correction
//     weights come from a first-order expansion around the tile's reference delay (exact
//     weights where the integer index differs from the reference).
// The default tile makes the link span (tile + halo) exactly one pass of the CTA's threads.
#include <cuda_runtime.h>

#include "lr_device.cuh"
#include "lr_mixed.cuh"
#include "lr_tdi_table.cuh"

namespace lr {

__constant__ TdiTab c_tdimx = make_tdi_tab();

constexpr int NTERM = 42;  // 3 channels x 2 chains x 7 delayed terms
constexpr float TAU_UNIT = 0x1p-10f;
constexpr float ETA = 0x1p-8f;  // half step of the central difference of the correction weights

struct MxShared {
    TileInfo ti;
    SkyConst sk;
    int64_t k_lo, w_lo;
    int ny, wlen;
    double u0;
    double scale, unscale;
    unsigned long long maxbits;
    // reading positions (window-local, fixed point) as cubics in the knot coordinate
    double rp[2][9][4];
    double xa[2];
    double rstep;
    int jsw;
    // TDI delays (fixed point samples) as cubics, over the output tile
    double dp[2][6][4];
    double xta[2];
    double rstep_t;
    int jswt;
    // geometry factors c+_l, cx_l as cubics in tau = (j - jc) 2^-10
    double gnode[4][12];
    double tmax;
    float g0h[12], g0l[12], g1h[12], g1l[12], g2[12], g3[12];
    int jc;
    // TDI reference per term
    int tfm[NTERM];
    float tehi[NTERM], telo[NTERM];
};

// ---------------------------------------------------------------- per-tile setup helpers
__device__ inline const double *orbit_coef_ptr(const OrbitDev &o, int K, int s)
{
    return o.coef + ((size_t)K * NSERIES + s) * 4;
}

__device__ inline int clampK(const OrbitDev &o, double u)
{
    double f = floor(u);
    int K = (int)f;
    return K < 0 ? 0 : (K > o.nint - 1 ? o.nint - 1 : K);
}

__device__ inline double horner3(const double *c, double x) { return fma(x, fma(x, fma(x, c[3], c[2]), c[1]), c[0]); }

// float-float value of a fitted geometry factor at tau
__device__ __forceinline__ ff geom_at(const MxShared &sh, int f, float tau)
{
    ff c = ff_add({sh.g0h[f], sh.g0l[f]}, ff_mul_f({sh.g1h[f], sh.g1l[f]}, tau));
    return ff_add_f(c, tau * tau * fmaf(tau, sh.g3[f], sh.g2[f]));
}

// Difference tables from float-float values held in S.shi / S.slo.  Entries whose difference
// stencils leave the window are set to 0 (they are never read).
__device__ void build_tables_ff(int len, const CompSeries &S)
{
    for (int j = threadIdx.x; j < len; j += blockDim.x) {
        ff s0 = {S.shi[j], S.slo[j]};
        float dh = 0.0f, dl = 0.0f, a = 0.0f, al = 0.0f, e = 0.0f;
        if (j + 1 < len) {
            ff s1 = {S.shi[j + 1], S.slo[j + 1]};
            ff d1 = ff_sub(s1, s0);
            dh = d1.hi;
            dl = d1.lo;
            if (j >= 1) {
                ff sm = {S.shi[j - 1], S.slo[j - 1]};
                ff dd = ff_sub(d1, ff_sub(s0, sm));
                a = 0.5f * dd.hi;
                al = 0.5f * dd.lo;
            }
            if (j + 3 < len) {
                ff s2 = {S.shi[j + 2], S.slo[j + 2]}, s3 = {S.shi[j + 3], S.slo[j + 3]};
                ff d2 = ff_sub(s2, s1), d3 = ff_sub(s3, s2);
                ff e3 = ff_sub(ff_sub(d3, d2), ff_sub(d2, d1));
                e = e3.hi + e3.lo;
            }
        }
        S.dhi[j] = dh;
        S.dlo[j] = dl;
        S.e[j] = e;
        if (S.alo) {
            S.a[j] = a;
            S.alo[j] = al;
        } else {
            S.a[j] = a + al;
        }
    }
}

// link-series tables: 6 arrays of `stride` floats; strain tables add the low part of a (7 arrays)
__device__ inline CompSeries series_at(float *base, int stride, bool with_alo = false)
{
    CompSeries S;
    S.shi = base;
    S.slo = base + stride;
    S.dhi = base + 2 * stride;
    S.dlo = base + 3 * stride;
    S.a = base + 4 * stride;
    S.e = base + 5 * stride;
    S.alo = with_alo ? base + 6 * stride : nullptr;
    return S;
}

// block max of |v| as the bit pattern of a non-negative double
__device__ inline void block_absmax(unsigned long long *dst, double v)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(fabs(v));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long c = __shfl_xor_sync(0xffffffffu, b, o);
        b = c > b ? c : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(dst, b);
}

__device__ inline void set_scale(MxShared &sh)
{
    double mx = __longlong_as_double((long long)sh.maxbits);
    if (mx > 0.0 && isfinite(mx)) {
        int E;
        frexp(mx, &E);
        sh.scale = ldexp(1.0, -E);
        sh.unscale = ldexp(1.0, E);
    } else {
        sh.scale = 1.0;
        sh.unscale = 1.0;
    }
}

// ---------------------------------------------------------------- setup phases
// Read-position cubics (threads 0..17), knot bookkeeping (thread 18) and geometry nodes
// (threads 32..43: node = i / 3, arm = i % 3).
__device__ void setup_projection(const FwdParams &P, MxShared &sh)
{
    const int tid = threadIdx.x;
    const OrbitDev &o = P.po;
    const double ua = (P.t0 + (double)sh.k_lo * P.dt - o.t_first) * o.inv_dk;
    const double ub = ua + (double)(sh.ny - 1) * P.dt * o.inv_dk;
    const int K0 = clampK(o, ua), K1 = clampK(o, ub);
    if (tid < 18) {
        const int iv = tid / 9, rd = tid % 9;
        const int K = iv == 0 ? K0 : K1;
        // emission reads (rd >= 3) of link l = rd - 3 shift by the emitter's k.x/c and L_l;
        // reception reads by the receiver's k.x/c
        const int sc = rd < 3 ? rd : (rd == 3 ? 1 : rd == 4 ? 2 : rd == 5 ? 0 : rd == 6 ? 2 : rd == 7 ? 1 : 0);
        double c[4] = {0.0, 0.0, 0.0, 0.0};
        const double kc = 1.0 / (C_LIGHT * P.dt);
        for (int d = 0; d < 3; ++d) {
            const double *q = orbit_coef_ptr(o, K, 3 * sc + d);
            for (int i = 0; i < 4; ++i) c[i] = fma(sh.sk.k[d] * kc, q[i], c[i]);
        }
        if (rd >= 3) {
            const double *q = orbit_coef_ptr(o, K, 9 + rd - 3);
            for (int i = 0; i < 4; ++i) c[i] = fma(q[i], P.inv_dt, c[i]);
        }
        const double base = (double)(sh.k_lo - sh.w_lo) + sh.u0;
        sh.rp[iv][rd][0] = (base - c[0]) * FX_ONE;
        for (int i = 1; i < 4; ++i) sh.rp[iv][rd][i] = -c[i] * FX_ONE;
    } else if (tid == 18) {
        sh.xa[0] = ua - (double)K0;
        sh.xa[1] = ua - (double)K1;
        sh.rstep = P.dt * o.inv_dk;
        int jsw = sh.ny;
        if (K1 != K0) {
            double jj = ceil(((double)K1 - ua) / sh.rstep);
            jsw = jj < 0 ? 0 : (jj > sh.ny ? sh.ny : (int)jj);
        }
        sh.jsw = jsw;
        sh.jc = sh.ny / 2;
        sh.tmax = ((double)(sh.ny / 2) + 1.0) * (double)TAU_UNIT;
    } else if (tid >= 32 && tid < 44) {
        // geometry factors of arm a at Chebyshev node i (Eq. projected-strain-ssb patterns,
        // psi rotation, 1/(2(1 -+ k.n)) for the two directions)
        const int i = (tid - 32) / 3, a = (tid - 32) % 3;
        const double tmax = ((double)(sh.ny / 2) + 1.0) * (double)TAU_UNIT;
        const double tau = tmax * cos((2.0 * i + 1.0) * 3.14159265358979323846 / 8.0);
        const double t = P.t0 + ((double)(sh.k_lo + sh.ny / 2) + tau / (double)TAU_UNIT) * P.dt;
        double x;
        const Coef4 *row = spline_row(o, t, &x);
        const int r = a, s = (a + 1) % 3;
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = cubic(ldg4(row + 3 * r + c), x) - cubic(ldg4(row + 3 * s + c), x);
        const SkyConst &S = sh.sk;
        double inv = 1.0 / sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double n0 = d[0] * inv, n1 = d[1] * inv, n2 = d[2] * inv;
        double un = S.u[0] * n0 + S.u[1] * n1 + S.u[2] * n2;
        double vn = S.v[0] * n0 + S.v[1] * n1 + S.v[2] * n2;
        double kn = S.k[0] * n0 + S.k[1] * n1 + S.k[2] * n2;
        double xip = un * un - vn * vn, xic = 2.0 * un * vn;
        double xp = S.c2p * xip + S.s2p * xic, xc = -S.s2p * xip + S.c2p * xic;
        double df = 0.5 / (1.0 - kn), dr = 0.5 / (1.0 + kn);
        sh.gnode[i][a] = xp * df;
        sh.gnode[i][6 + a] = xc * df;
        sh.gnode[i][5 - a] = xp * dr;
        sh.gnode[i][11 - a] = xc * dr;
    }
}

// cubic through the 4 geometry nodes: monomial coefficients in tau from the Chebyshev
// inverse Vandermonde (threads 64..75)
__device__ void fit_geometry(const FwdParams &P, MxShared &sh)
{
    const int f = threadIdx.x - 64;
    if (f < 0 || f >= 12) return;
    double b[4];
    double sc = 1.0;
    for (int k = 0; k < 4; ++k) {
        double acc = 0.0;
        for (int i = 0; i < 4; ++i) acc = fma(P.cheb[k][i], sh.gnode[i][f], acc);
        b[k] = acc * sc;
        sc /= sh.tmax;
    }
    ff c0 = ff_from_double(b[0]), c1 = ff_from_double(b[1]);
    sh.g0h[f] = c0.hi; sh.g0l[f] = c0.lo;
    sh.g1h[f] = c1.hi; sh.g1l[f] = c1.lo;
    sh.g2[f] = (float)b[2];
    sh.g3[f] = (float)b[3];
}

// TDI delay cubics over the output tile (fixed point, samples x 2^44): threads 96..107, 108
__device__ void setup_tdi(const FwdParams &P, MxShared &sh, int64_t n0, int nb)
{
    const int tid = threadIdx.x;
    const OrbitDev &o = P.to;
    const double ua = (P.t0 + (double)n0 * P.dt - o.t_first) * o.inv_dk;
    const double ub = ua + (double)(nb > 0 ? nb - 1 : 0) * P.dt * o.inv_dk;
    const int K0 = clampK(o, ua), K1 = clampK(o, ub);
    if (tid >= 96 && tid < 108) {
        const int iv = (tid - 96) / 6, l = (tid - 96) % 6;
        const double *q = orbit_coef_ptr(o, iv == 0 ? K0 : K1, 9 + l);
        for (int i = 0; i < 4; ++i) sh.dp[iv][l][i] = q[i] * P.inv_dt * FX_ONE;
    } else if (tid == 108) {
        sh.xta[0] = ua - (double)K0;
        sh.xta[1] = ua - (double)K1;
        sh.rstep_t = P.dt * o.inv_dk;
        int jsw = nb;
        if (K1 != K0) {
            double jj = ceil(((double)K1 - ua) / sh.rstep_t);
            jsw = jj < 0 ? 0 : (jj > nb ? nb : (int)jj);
        }
        sh.jswt = jsw;
    }
}

// fixed-point delays (samples x 2^44) of the six links at output index i of the tile
__device__ __forceinline__ void tdi_delays_fx(const MxShared &sh, int i, long long &L0, long long &L1, long long &L2,
                                              long long &L3, long long &L4, long long &L5)
{
    const int iv = i < sh.jswt ? 0 : 1;
    const double x = fma((double)i, sh.rstep_t, sh.xta[iv]);
    L0 = __double2ll_rn(horner3(sh.dp[iv][0], x));
    L1 = __double2ll_rn(horner3(sh.dp[iv][1], x));
    L2 = __double2ll_rn(horner3(sh.dp[iv][2], x));
    L3 = __double2ll_rn(horner3(sh.dp[iv][3], x));
    L4 = __double2ll_rn(horner3(sh.dp[iv][4], x));
    L5 = __double2ll_rn(horner3(sh.dp[iv][5], x));
}

__device__ __forceinline__ long long pick(int l, long long L0, long long L1, long long L2, long long L3, long long L4,
                                          long long L5)
{
    return l == 0 ? L0 : l == 1 ? L1 : l == 2 ? L2 : l == 3 ? L3 : l == 4 ? L4 : L5;
}

// Per-tile reference of each delayed TDI term at the tile centre, and its correction weights at
// eps_ref - ETA, eps_ref, eps_ref + ETA (threads 128..253: term = i / 3, point = i % 3).
template <int T>
__device__ void setup_tdi_refs(const FwdParams &P, MxShared &sh, int nb, float *tw)
{
    constexpr int NU = T >= 4 ? T - 3 : 1;
    const int i = threadIdx.x - 128;
    if (i < 0 || i >= 3 * NTERM) return;
    const int id = i / 3, pt = i % 3;
    const int ch = id / 14, c = (id / 7) % 2, q = id % 7 + 1;
    if (q > P.q_terms) return;
    long long L0, L1, L2, L3, L4, L5;
    tdi_delays_fx(sh, nb / 2, L0, L1, L2, L3, L4, L5);
    long long D = 0;
    for (int k = 1; k <= q; ++k) D += pick(chain_pair(ch, c, k), L0, L1, L2, L3, L4, L5);
    Split s = split_fx(-D);
    if (pt == 1) {
        sh.tfm[id] = s.m;
        sh.tehi[id] = s.ehi;
        sh.telo[id] = s.elo;
    }
    if constexpr (T >= 4) {
        float U[NU];
        comp_weights<T>(s.ehi + (float)(pt - 1) * ETA, U);
        float *w = tw + ((size_t)id * 3 + pt) * NU;
#pragma unroll
        for (int a = 0; a < NU; ++a) w[a] = U[a];
    }
}

// [U(eps - ETA), U(eps), U(eps + ETA)] -> [U(eps), dU/deps] in place
template <int T>
__device__ void finish_tdi_refs(const FwdParams &P, float *tw)
{
    constexpr int NU = T >= 4 ? T - 3 : 1;
    if constexpr (T >= 4) {
        for (int idx = threadIdx.x; idx < NTERM * NU; idx += blockDim.x) {
            const int id = idx / NU, a = idx % NU;
            if (id % 7 + 1 > P.q_terms) continue;
            float *w = tw + (size_t)id * 3 * NU;
            float um = w[a], u0 = w[NU + a], up = w[2 * NU + a];
            w[a] = u0;
            w[NU + a] = (up - um) * (0.5f / ETA);
        }
    }
}

// ---------------------------------------------------------------- per-sample work
// One compensated read of both polarisations at read `rd` (0-2: reception at spacecraft rd,
// 3-8: emission of link rd-3) for y-local index j.  A stencil outside the staged window records
// ERR_WINDOW and reads as zero.
template <int T>
__device__ __forceinline__ void strain_read(const MxShared &sh, const CompSeries &Hp, const CompSeries &Hc, int iv,
                                            double x, long long jfx, int rd, int *err, ff &vp, ff &vc)
{
    constexpr int NU = T >= 4 ? T - 3 : 1;
    constexpr int h = (T - 2) / 2;
    long long X = __double2ll_rn(horner3(sh.rp[iv][rd], x)) + jfx;
    Split s = split_fx(X);
    if (s.m - h < 0 || s.m + h + 1 >= sh.wlen) {
        atomicOr(err, ERR_WINDOW);
        vp = vc = {0.0f, 0.0f};
        return;
    }
    float U[NU];
    if constexpr (T >= 4) comp_weights<T>(s.ehi, U);
    vp = comp_value<T, true>(Hp, s.m, s.ehi, s.elo, U);
    vc = comp_value<T, true>(Hc, s.m, s.ehi, s.elo, U);
}

// Six link samples (scaled, float-float) at y-local index j, handed to store(l, value):
// y_l = c+_l (h+(emission) - h+(reception)) + cx_l (hx(emission) - hx(reception)).
template <int T, class Store>
__device__ void project_sample_mx(const MxShared &sh, const CompSeries &Hp, const CompSeries &Hc, int j, int *err,
                                  Store store)
{
    const int iv = j < sh.jsw ? 0 : 1;
    const double x = fma((double)j, sh.rstep, sh.xa[iv]);
    const long long jfx = (long long)j << FX_BITS;
    ff Rp0, Rp1, Rp2, Rc0, Rc1, Rc2;
    strain_read<T>(sh, Hp, Hc, iv, x, jfx, 0, err, Rp0, Rc0);
    strain_read<T>(sh, Hp, Hc, iv, x, jfx, 1, err, Rp1, Rc1);
    strain_read<T>(sh, Hp, Hc, iv, x, jfx, 2, err, Rp2, Rc2);
    const float tau = (float)(j - sh.jc) * TAU_UNIT;
#pragma unroll 1
    for (int l = 0; l < 6; ++l) {
        ff ep, ec;
        strain_read<T>(sh, Hp, Hc, iv, x, jfx, 3 + l, err, ep, ec);
        const int r = l < 3 ? l : (l == 3 ? 0 : (l == 4 ? 2 : 1));   // receiving spacecraft
        const ff rp = r == 0 ? Rp0 : (r == 1 ? Rp1 : Rp2);
        const ff rc = r == 0 ? Rc0 : (r == 1 ? Rc1 : Rc2);
        store(l, ff_add(ff_mul(geom_at(sh, l, tau), ff_sub(ep, rp)), ff_mul(geom_at(sh, 6 + l, tau), ff_sub(ec, rc))));
    }
}

// exact-weight read of a link series (used where the integer index differs from the tile's
// reference): kept out of line, it is rare
template <int T>
__device__ __noinline__ ff link_read_exact(const CompSeries S, int m, float ehi, float elo)
{
    constexpr int NU = T >= 4 ? T - 3 : 1;
    float U[NU];
    if constexpr (T >= 4) comp_weights<T>(ehi, U);
    return comp_value<T>(S, m, ehi, elo, U);
}

// X, Y, Z of one output sample: for each channel the two Michelson chains, each a running
// fixed-point delay over the chain's links; every delayed read uses the tile-reference expansion
// of its correction weights unless its integer index differs from the reference.
template <int T>
__device__ __forceinline__ void tdi_sample_mx(const FwdParams &P, const MxShared &sh, float *ybase, int ystride, int nl,
                                              const float *tw, long long L0, long long L1, long long L2, long long L3,
                                              long long L4, long long L5, double *o, int64_t N, double us)
{
    constexpr int NU = T >= 4 ? T - 3 : 1;
    constexpr int h = (T - 2) / 2;
    const long long nlfx = (long long)nl << FX_BITS;
#pragma unroll 1
    for (int ch = 0; ch < 3; ++ch) {
        ff acc = {0.0f, 0.0f};
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
            const int l0 = c_tdimx.link[ch][c][0];
            ff part = {ybase[(6 * l0 + 0) * ystride + nl], ybase[(6 * l0 + 1) * ystride + nl]};
            long long D = 0;
#pragma unroll 1
            for (int q = 1; q <= P.q_terms; ++q) {
                D += pick(c_tdimx.pair[ch][c][q], L0, L1, L2, L3, L4, L5);
                const int lk = c_tdimx.link[ch][c][q];
                const int id = (ch * 2 + c) * 7 + (q - 1);
                CompSeries S = series_at(ybase + 6 * lk * ystride, ystride);
                Split s = split_fx(nlfx - D);
                ff v;
                if (s.m - h < 0 || s.m + h + 1 >= sh.ny) {
                    atomicOr(P.err, ERR_WINDOW);
                    v = {0.0f, 0.0f};
                } else if (s.m - nl == sh.tfm[id]) {
                    const float delta = (s.ehi - sh.tehi[id]) + (s.elo - sh.telo[id]);
                    const float *w0 = tw + (size_t)id * 3 * NU;
                    v = comp_value_taylor<T>(S, s.m, s.ehi, s.elo, w0, w0 + NU, delta);
                } else {
                    v = link_read_exact<T>(S, s.m, s.ehi, s.elo);
                }
                part = ff_add(part, v);
            }
            acc = c == 0 ? part : ff_sub(acc, part);
        }
        o[ch * N] = ff_to_double(acc) * us;
    }
}

// ---------------------------------------------------------------- kernels
// Shared memory (floats): [strain tables 14 W][link tables 36 Y (also the FP64 staging
// buffer, 4 W floats)][TDI correction weights 3*42*(T-3)].
__host__ __device__ inline void mx_layout(const FwdParams &P, int T, size_t *r2, size_t *r3, size_t *total)
{
    const size_t W = (size_t)P.wmax, Y = (size_t)P.ymax;
    size_t a = 14 * W;
    size_t b = 36 * Y > 4 * W ? 36 * Y : 4 * W;
    if (12 * Y > a) a = 12 * Y;  // TDI-only launches stage FP64 link series in region 1
    size_t c = 3 * NTERM * (size_t)(T >= 4 ? T - 3 : 1);
    *r2 = a;
    *r3 = a + b;
    *total = a + b + c;
}

template <int T, int KIND>
__global__ void __launch_bounds__(256, 2) k_mixed(FwdParams P)
{
    extern __shared__ float smf[];
    __shared__ MxShared sh;
    size_t r2, r3, total;
    mx_layout(P, T, &r2, &r3, &total);
    float *R1 = smf, *R2 = smf + r2, *tw = smf + r3;
    const int W = P.wmax, Y = P.ymax;
    CompSeries Hp = series_at(R1, W, true), Hc = series_at(R1 + 7 * W, W, true);
    const int64_t tot = P.total_tiles >= 0 ? P.total_tiles : P.src.tile_off[P.src.S];
    for (int64_t g = blockIdx.x; g < tot; g += gridDim.x) {
        if (threadIdx.x == 0) {
            sh.ti = tile_info(P, g, KIND == KIND_PROJECT ? 6 : 3);
            sh.sk = make_sky(sh.ti.sky);
            if (!sh.ti.ok) atomicOr(P.err, ERR_OFFSETS);
            const int hl = KIND == KIND_PROJECT ? 0 : P.HL, hr = KIND == KIND_PROJECT ? 0 : P.HR;
            sh.k_lo = sh.ti.n0 - hl;
            sh.ny = (int)sh.ti.nb + hl + hr;
            sh.u0 = (P.t0 - sh.ti.t0h) / P.dt;
            const int h = (T - 2) / 2;
            sh.w_lo = sh.k_lo + (int64_t)floor(sh.u0) - P.sig_b - P.lproj_b - h - 2;
            sh.wlen = sh.ny + 2 * P.sig_b + P.lproj_b + T + 4;
            sh.maxbits = 0ull;
        }
        __syncthreads();
        if (!sh.ti.ok || sh.ti.nb <= 0) {
            __syncthreads();
            continue;
        }
        const int ny = sh.ny, nb = (int)sh.ti.nb;
        // ---- phase 1: stage raw inputs and their max; per-tile cubics and geometry nodes
        if (KIND != KIND_TDI) {
            double *tmp = reinterpret_cast<double *>(R2);
            double mx = 0.0;
            for (int j = threadIdx.x; j < sh.wlen; j += blockDim.x) {
                int64_t i = sh.w_lo + j;
                bool in = i >= 0 && i < sh.ti.nh;
                double a = in ? __ldg(sh.ti.hp + i) : 0.0, b = in ? __ldg(sh.ti.hc + i) : 0.0;
                tmp[j] = a;
                tmp[W + j] = b;
                mx = fmax(mx, fmax(fabs(a), fabs(b)));
            }
            block_absmax(&sh.maxbits, mx);
            setup_projection(P, sh);
        } else {
            double *tmp = reinterpret_cast<double *>(R1);
            double mx = 0.0;
            for (int l = 0; l < 6; ++l)
                for (int j = threadIdx.x; j < ny; j += blockDim.x) {
                    int64_t k = sh.k_lo + j;
                    double v = (k >= 0 && k < sh.ti.N) ? __ldg(sh.ti.yin + l * sh.ti.N + k) : 0.0;
                    tmp[l * Y + j] = v;
                    mx = fmax(mx, fabs(v));
                }
            block_absmax(&sh.maxbits, mx);
        }
        if (KIND != KIND_PROJECT) setup_tdi(P, sh, sh.ti.n0, nb);
        __syncthreads();
        // ---- phase 2: scale, geometry fits, TDI reference weights
        if (threadIdx.x == 0) set_scale(sh);
        if (KIND != KIND_TDI) fit_geometry(P, sh);
        if (KIND != KIND_PROJECT) setup_tdi_refs<T>(P, sh, nb, tw);
        __syncthreads();
        // ---- phase 3: scaled float-float values
        if (KIND != KIND_TDI) {
            const double *tmp = reinterpret_cast<const double *>(R2);
            for (int j = threadIdx.x; j < sh.wlen; j += blockDim.x) {
                ff a = ff_from_double(tmp[j] * sh.scale), b = ff_from_double(tmp[W + j] * sh.scale);
                Hp.shi[j] = a.hi; Hp.slo[j] = a.lo;
                Hc.shi[j] = b.hi; Hc.slo[j] = b.lo;
            }
        } else {
            const double *tmp = reinterpret_cast<const double *>(R1);
            for (int l = 0; l < 6; ++l)
                for (int j = threadIdx.x; j < ny; j += blockDim.x) {
                    ff v = ff_from_double(tmp[l * Y + j] * sh.scale);
                    R2[(6 * l + 0) * Y + j] = v.hi;
                    R2[(6 * l + 1) * Y + j] = v.lo;
                }
        }
        if (KIND != KIND_PROJECT) finish_tdi_refs<T>(P, tw);
        __syncthreads();
        // ---- phase 4/5: strain difference tables, link series
        if (KIND != KIND_TDI) {
            build_tables_ff(sh.wlen, Hp);
            build_tables_ff(sh.wlen, Hc);
            __syncthreads();
            for (int j = threadIdx.x; j < ny; j += blockDim.x) {
                const int64_t k = sh.k_lo + j;
                const bool in = k >= 0 && k < sh.ti.N;
                if (KIND == KIND_PROJECT) {
                    double *o = sh.ti.out;
                    const int64_t N = sh.ti.N;
                    const double us = sh.unscale;
                    project_sample_mx<T>(sh, Hp, Hc, j, P.err,
                                         [&](int l, ff v) { o[l * N + k] = ff_to_double(v) * us; });
                } else if (in) {
                    project_sample_mx<T>(sh, Hp, Hc, j, P.err, [&](int l, ff v) {
                        R2[(6 * l + 0) * Y + j] = v.hi;
                        R2[(6 * l + 1) * Y + j] = v.lo;
                    });
                } else {
#pragma unroll
                    for (int l = 0; l < 6; ++l) {
                        R2[(6 * l + 0) * Y + j] = 0.0f;
                        R2[(6 * l + 1) * Y + j] = 0.0f;
                    }
                }
            }
        }
        // ---- phase 6/7: link difference tables, X, Y, Z
        if (KIND != KIND_PROJECT) {
            __syncthreads();
            for (int l = 0; l < 6; ++l) build_tables_ff(ny, series_at(R2 + 6 * l * Y, Y));
            __syncthreads();
            for (int i = threadIdx.x; i < nb; i += blockDim.x) {
                const int64_t n = sh.ti.n0 + i;
                const int nl = (int)(n - sh.k_lo);
                long long L0, L1, L2, L3, L4, L5;
                tdi_delays_fx(sh, i, L0, L1, L2, L3, L4, L5);
                tdi_sample_mx<T>(P, sh, R2, Y, nl, tw, L0, L1, L2, L3, L4, L5, sh.ti.out + n, sh.ti.N, sh.unscale);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- dispatch
template <int T>
static void *kernel_ptr_mx(int kind)
{
    switch (kind) {
        case KIND_PROJECT: return (void *)k_mixed<T, KIND_PROJECT>;
        case KIND_TDI: return (void *)k_mixed<T, KIND_TDI>;
        default: return (void *)k_mixed<T, KIND_FUSED>;
    }
}

#define LR_MX_ORDERS(X) X(1) X(3) X(5) X(7) X(9) X(11) X(13) X(15) X(17) X(19) X(21) X(23) X(25) X(31) X(41)

static void *kernel_for_mx(int kind, int order)
{
    switch (order) {
#define LR_CASE(p) case p: return kernel_ptr_mx<p + 1>(kind);
        LR_MX_ORDERS(LR_CASE)
#undef LR_CASE
        default: return nullptr;
    }
}

int smem_fwdmx(int kind, int order, const FwdParams &P, size_t *smem)
{
    (void)kind;
    size_t r2, r3, total;
    mx_layout(P, order + 1, &r2, &r3, &total);
    *smem = total * sizeof(float);
    return 0;
}

int max_blocks_fwdmx(int kind, int order, int threads, size_t smem, int *blocks)
{
    void *k = kernel_for_mx(kind, order);
    if (!k) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, threads, smem);
}

int launch_fwdmx(int kind, int order, const FwdParams &P, int grid, int threads, size_t smem, void *stream)
{
    void *k = kernel_for_mx(kind, order);
    if (!k) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    void *args[] = {(void *)&P};
    return (int)cudaLaunchKernel(k, dim3(grid), dim3(threads), args, smem, (cudaStream_t)stream);
}

bool order_compiled_mx(int order) { return kernel_for_mx(KIND_FUSED, order) != nullptr; }

}  // namespace lr
