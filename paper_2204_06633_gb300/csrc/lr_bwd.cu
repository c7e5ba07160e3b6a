// Backward (adjoint) kernels: the transpose of the response applied to dLoss/dXYZ.
//
//   K1  g_y  = T^T g_xyz   tile over link samples k; for every delayed TDI term the CTA writes
//                           the Lagrange weights of each output n in the tile's window to shared
//                           memory, then every thread gathers the taps that land on its k
//                           (the inverted tap window): deterministic, no atomics on data.
//   K2  g_h  = P^T g_y     tile over strain samples i; for each of the 9 reads (3 receptions,
//                           6 emissions) the weights of every link sample in the tile's window,
//                           then a gather onto i for both polarisations.
//   K3  dLoss/d(lambda, beta, psi) partial sums per tile: the derivative of each link sample
//                           (patterns, 1/(1 - k.n) and read times through k) against g_y,
//                           with derivative Lagrange weights; K4 adds the partials in order.
// All arithmetic is FP64.  Link series are never stored: K1 only needs the orbit, K3 recomputes
// the strain reads.
#include <cuda_runtime.h>

#include "lr_bwd.h"
#include "lr_device.cuh"
#include "lr_tdi_table.cuh"

namespace lr {

__constant__ TdiTab c_tdibw = make_tdi_tab();

// ---------------------------------------------------------------- weights
// explicit centered Lagrange weights w_a = (-1)^(T-1-a) L_a R_a (prefix and suffix products)
template <int T>
__device__ __forceinline__ void lagrange_w64(double e, double *w)
{
    constexpr int h = (T - 2) / 2;
    double L = 1.0;
#pragma unroll
    for (int a = 0; a < T; ++a) {
        w[a] = L;
        L *= fma(e, 1.0 / (double)(a + 1), (double)(h - a) / (double)(a + 1));
    }
    double R = 1.0;
#pragma unroll
    for (int a = T - 1; a >= 0; --a) {
        const double sg = ((T - 1 - a) & 1) ? -1.0 : 1.0;
        w[a] = sg * w[a] * R;
        R *= fma(e, 1.0 / (double)(T - a), (double)(h - a) / (double)(T - a));
    }
}

// weights and their derivatives dw/deps (product rule through the prefix and suffix products)
template <int T>
__device__ __forceinline__ void lagrange_wd64(double e, double *w, double *dw)
{
    constexpr int h = (T - 2) / 2;
    double L = 1.0, dL = 0.0;
#pragma unroll
    for (int a = 0; a < T; ++a) {
        w[a] = L;
        dw[a] = dL;
        const double k1 = 1.0 / (double)(a + 1);
        const double f = fma(e, k1, (double)(h - a) * k1);
        dL = fma(dL, f, L * k1);
        L *= f;
    }
    double R = 1.0, dR = 0.0;
#pragma unroll
    for (int a = T - 1; a >= 0; --a) {
        const double sg = ((T - 1 - a) & 1) ? -1.0 : 1.0;
        const double nw = sg * w[a] * R;
        dw[a] = sg * fma(dw[a], R, w[a] * dR);
        w[a] = nw;
        const double k1 = 1.0 / (double)(T - a);
        const double f = fma(e, k1, (double)(h - a) * k1);
        dR = fma(dR, f, R * k1);
        R *= f;
    }
}

__device__ __forceinline__ void add_to(double *acc, int l, double v)
{
#pragma unroll
    for (int i = 0; i < 6; ++i)
        if (i == l) acc[i] += v;
}

// ---------------------------------------------------------------- K1: TDI transpose
// Shared memory (doubles): G[3][WN] (g_xyz window), Ls[6][WN] (delays / dt), W[T][WN]
// (weights of the current term); ints Mo[WN] (floor of the read offset).
template <int T>
__global__ void __launch_bounds__(256) k_tdi_adj64(FwdParams P, BwdParams B)
{
    constexpr int h = (T - 2) / 2;
    extern __shared__ double sm[];
    const int WN = B.wn;
    double *G = sm, *Ls = sm + 3 * WN, *W = sm + 9 * WN;
    int *Mo = reinterpret_cast<int *>(sm + (9 + T) * WN);
    __shared__ TileInfo ti;
    __shared__ int mo_lo, mo_hi;
    const int64_t total = P.total_tiles >= 0 ? P.total_tiles : P.src.tile_off[P.src.S];
    for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
        if (threadIdx.x == 0) {
            ti = tile_info(P, g, 3);
            if (!ti.ok) atomicOr(P.err, ERR_OFFSETS);
        }
        __syncthreads();
        if (!ti.ok || ti.nb <= 0) {
            __syncthreads();
            continue;
        }
        const int64_t N = ti.N, k0 = ti.n0, n_lo = k0 - h - 2;
        const int nb = (int)ti.nb, wn = nb + 2 * h + 5 + B.dmax;
        const double *gx = B.g_xyz + (ti.out - P.out);   // same source offset as the outputs
        for (int j = threadIdx.x; j < wn; j += blockDim.x) {
            const int64_t n = n_lo + j;
            const bool in = n >= 0 && n < N;
            for (int c = 0; c < 3; ++c) G[c * WN + j] = in ? __ldg(gx + c * N + n) : 0.0;
            double L[6];
            orbit_delays(P.to, P.t0 + (double)n * P.dt, L);
            for (int l = 0; l < 6; ++l) Ls[l * WN + j] = L[l] * P.inv_dt;
        }
        double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        const int me = threadIdx.x;
        const int64_t k = k0 + me;
        __syncthreads();
        if (me < nb) {
            for (int ch = 0; ch < 3; ++ch) {
                const double gv = G[ch * WN + (int)(k - n_lo)];
                add_to(acc, c_tdibw.link[ch][0][0], gv);
                add_to(acc, c_tdibw.link[ch][1][0], -gv);
            }
        }
        for (int ch = 0; ch < 3; ++ch)
            for (int c = 0; c < 2; ++c)
                for (int q = 1; q <= P.q_terms; ++q) {
                    if (threadIdx.x == 0) {
                        mo_lo = 1 << 30;
                        mo_hi = -(1 << 30);
                    }
                    __syncthreads();
                    int lmin = 1 << 30, lmax = -(1 << 30);
                    for (int j = threadIdx.x; j < wn; j += blockDim.x) {
                        double D = 0.0;
                        if (P.delay_nested) {
                            const double t = P.t0 + (double)(n_lo + j) * P.dt;
                            for (int qq = 1; qq <= q; ++qq) D += orbit_delay1(P.to, t - D, c_tdibw.pair[ch][c][qq]);
                            D *= P.inv_dt;
                        } else {
                            for (int qq = 1; qq <= q; ++qq) D += Ls[c_tdibw.pair[ch][c][qq] * WN + j];
                        }
                        const double u = -D, fl = floor(u);
                        const int mo = (int)fl;
                        Mo[j] = mo;
                        lmin = min(lmin, mo);
                        lmax = max(lmax, mo);
                        double w[T];
                        lagrange_w64<T>(u - fl, w);
#pragma unroll
                        for (int a = 0; a < T; ++a) W[a * WN + j] = w[a];
                    }
                    atomicMin(&mo_lo, lmin);
                    atomicMax(&mo_hi, lmax);
                    __syncthreads();
                    if (me < nb) {
                        // outputs n whose stencil [n + Mo - h, n + Mo + h + 1] contains k
                        int jlo = (int)(k - h - 1 - mo_hi - n_lo), jhi = (int)(k + h - mo_lo - n_lo);
                        jlo = max(jlo, 0);
                        jhi = min(jhi, wn - 1);
                        double s = 0.0;
                        for (int j = jlo; j <= jhi; ++j) {
                            const int a = (int)(k - (n_lo + j + Mo[j])) + h;
                            if (a >= 0 && a < T) s = fma(W[a * WN + j], G[ch * WN + j], s);
                        }
                        add_to(acc, c_tdibw.link[ch][c][q], c == 0 ? s : -s);
                    }
                    __syncthreads();
                }
        if (me < nb) {
            double *gy = B.g_y + 6 * (ti.out - P.out) / 3;
#pragma unroll
            for (int l = 0; l < 6; ++l) gy[l * N + k] = acc[l];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- geometry helpers
struct LinkGeo {
    double xp, xc, kn, den;
};

// patterns (rotated by 2 psi), k.n and 1/(2(1 - k.n)) of link l from positions x[9]
__device__ __forceinline__ LinkGeo link_geo(const SkyConst &S, const double *x, int l, double *nvec)
{
    const int LR[6] = {0, 1, 2, 0, 2, 1}, LSd[6] = {1, 2, 0, 2, 1, 0};
    const int r = LR[l], s = LSd[l];
    double d0 = x[3 * r] - x[3 * s], d1 = x[3 * r + 1] - x[3 * s + 1], d2 = x[3 * r + 2] - x[3 * s + 2];
    double inv = 1.0 / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    d0 *= inv; d1 *= inv; d2 *= inv;
    nvec[0] = d0; nvec[1] = d1; nvec[2] = d2;
    double un = S.u[0] * d0 + S.u[1] * d1 + S.u[2] * d2;
    double vn = S.v[0] * d0 + S.v[1] * d1 + S.v[2] * d2;
    LinkGeo g;
    g.kn = S.k[0] * d0 + S.k[1] * d1 + S.k[2] * d2;
    double xip = un * un - vn * vn, xic = 2.0 * un * vn;
    g.xp = S.c2p * xip + S.s2p * xic;
    g.xc = -S.s2p * xip + S.c2p * xic;
    g.den = 1.0 / (2.0 * (1.0 - g.kn));
    return g;
}

// ---------------------------------------------------------------- K2: projection transpose
// Shared memory (doubles): U[9][WK] read positions, CF[18][WK] coefficients (read, pol),
// W[T][WK] weights of the current read; ints Mo[WK].
template <int T>
__global__ void __launch_bounds__(256) k_proj_adj64(FwdParams P, BwdParams B)
{
    constexpr int h = (T - 2) / 2;
    extern __shared__ double sm[];
    const int WK = B.wk;
    double *U = sm, *CF = sm + 9 * WK, *W = sm + 27 * WK;
    int *Mo = reinterpret_cast<int *>(sm + (27 + T) * WK);
    __shared__ TileInfo ti;
    __shared__ SkyConst skc;
    __shared__ int64_t i0s, k_lo_s;
    __shared__ int nbs, wks, mo_lo, mo_hi;
    __shared__ double u0s;
    const int64_t total = B.h_total_tiles >= 0 ? B.h_total_tiles : B.h_tile_off[P.src.S];
    for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
        if (threadIdx.x == 0) {
            // tile over strain samples: map g to its source through the strain tile table
            FwdParams Q = P;
            Q.src.tile_off = B.h_tile_off;
            Q.tile = B.tile_h;
            ti = tile_info(Q, g, 3);
            if (!ti.ok) atomicOr(P.err, ERR_OFFSETS);
            skc = make_sky(ti.sky);
            u0s = (P.t0 - ti.t0h) / P.dt;
        }
        __syncthreads();
        if (!ti.ok) {
            __syncthreads();
            continue;
        }
        if (threadIdx.x == 0) {
            // tile_info clipped the tile against the output count; the strain tile is clipped
            // against the strain length instead
            const int64_t i0 = ti.n0;
            const int64_t nbh = ti.nh - i0;
            nbs = (int)(nbh < B.tile_h ? (nbh > 0 ? nbh : 0) : B.tile_h);
            i0s = i0;
            // reads of link samples near k_ref = i0 - u0: their shifts bound the k-window
            const int64_t k_ref = i0 - (int64_t)floor(u0s);
            double x[9], L[6];
            orbit_all(P.po, P.t0 + (double)k_ref * P.dt, x, L);
            double umin = 1e300, umax = -1e300;
            for (int rd = 0; rd < 9; ++rd) {
                int sc = rd < 3 ? rd : (rd == 3 ? 1 : rd == 4 ? 2 : rd == 5 ? 0 : rd == 6 ? 2 : rd == 7 ? 1 : 0);
                double u = u0s - (skc.k[0] * x[3 * sc] + skc.k[1] * x[3 * sc + 1] + skc.k[2] * x[3 * sc + 2]) /
                                     C_LIGHT * P.inv_dt;
                if (rd >= 3) u -= L[rd - 3] * P.inv_dt;
                umin = fmin(umin, u);
                umax = fmax(umax, u);
            }
            k_lo_s = i0 - h - 2 - (int64_t)ceil(umax) - B.kmargin;
            int64_t k_hi = i0 + nbs + h + 1 - (int64_t)floor(umin) + B.kmargin;
            int64_t w = k_hi - k_lo_s;
            if (w > WK) {
                atomicOr(P.err, ERR_WINDOW);
                w = WK;
            }
            wks = (int)w;
        }
        __syncthreads();
        const int nb = nbs, wk = wks;
        const int64_t k_lo = k_lo_s, i0 = i0s, N = ti.N;
        if (nb <= 0) {
            __syncthreads();
            continue;
        }
        const double *gy = B.g_y + 6 * (ti.out - P.out) / 3;
        // coefficients of every read at every link sample of the window
        for (int j = threadIdx.x; j < wk; j += blockDim.x) {
            const int64_t k = k_lo + j;
            if (k < 0 || k >= N) {
                for (int rd = 0; rd < 9; ++rd) {
                    U[rd * WK + j] = u0s;
                    CF[(2 * rd) * WK + j] = 0.0;
                    CF[(2 * rd + 1) * WK + j] = 0.0;
                }
                continue;
            }
            double x[9], L[6];
            orbit_all(P.po, P.t0 + (double)k * P.dt, x, L);
            double sig[3];
            for (int i = 0; i < 3; ++i)
                sig[i] = (skc.k[0] * x[3 * i] + skc.k[1] * x[3 * i + 1] + skc.k[2] * x[3 * i + 2]) / C_LIGHT * P.inv_dt;
            double rp[3] = {0, 0, 0}, rc[3] = {0, 0, 0};
            for (int l = 0; l < 6; ++l) {
                const int LR[6] = {0, 1, 2, 0, 2, 1}, LSd[6] = {1, 2, 0, 2, 1, 0};
                double nv[3];
                LinkGeo q = link_geo(skc, x, l, nv);
                const double gl = __ldg(gy + l * N + k) * q.den;
                U[(3 + l) * WK + j] = u0s - L[l] * P.inv_dt - sig[LSd[l]];
                CF[(2 * (3 + l)) * WK + j] = gl * q.xp;
                CF[(2 * (3 + l) + 1) * WK + j] = gl * q.xc;
                rp[LR[l]] -= gl * q.xp;
                rc[LR[l]] -= gl * q.xc;
            }
            for (int r = 0; r < 3; ++r) {
                U[r * WK + j] = u0s - sig[r];
                CF[(2 * r) * WK + j] = rp[r];
                CF[(2 * r + 1) * WK + j] = rc[r];
            }
        }
        __syncthreads();
        const int me = threadIdx.x;
        const int64_t i = i0 + me;
        double ap = 0.0, ac = 0.0;
        for (int rd = 0; rd < 9; ++rd) {
            if (threadIdx.x == 0) {
                mo_lo = 1 << 30;
                mo_hi = -(1 << 30);
            }
            __syncthreads();
            int lmin = 1 << 30, lmax = -(1 << 30);
            for (int j = threadIdx.x; j < wk; j += blockDim.x) {
                const double u = U[rd * WK + j], fl = floor(u);
                const int mo = (int)fl;
                Mo[j] = mo;
                lmin = min(lmin, mo);
                lmax = max(lmax, mo);
                double w[T];
                lagrange_w64<T>(u - fl, w);
#pragma unroll
                for (int a = 0; a < T; ++a) W[a * WK + j] = w[a];
            }
            atomicMin(&mo_lo, lmin);
            atomicMax(&mo_hi, lmax);
            __syncthreads();
            if (me < nb) {
                // link samples k whose read stencil [k + Mo - h, k + Mo + h + 1] contains i
                int jlo = (int)(i - h - 1 - mo_hi - k_lo), jhi = (int)(i + h - mo_lo - k_lo);
                jlo = max(jlo, 0);
                jhi = min(jhi, wk - 1);
                for (int j = jlo; j <= jhi; ++j) {
                    const int a = (int)(i - (k_lo + j + Mo[j])) + h;
                    if (a >= 0 && a < T) {
                        const double wv = W[a * WK + j];
                        ap = fma(wv, CF[(2 * rd) * WK + j], ap);
                        ac = fma(wv, CF[(2 * rd + 1) * WK + j], ac);
                    }
                }
            }
            __syncthreads();
        }
        if (me < nb) {
            B.g_hp[(ti.hp - P.hp) + i] = ap;
            B.g_hc[(ti.hp - P.hp) + i] = ac;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- K3: sky-angle gradient
// value and derivative (d/dposition) of a staged series at base + u
template <int T>
__device__ __forceinline__ void read_vd(const double *sp, const double *sc, int64_t base, double u, int64_t w_lo,
                                        int wlen, int *err, double &vp, double &dp, double &vc, double &dc)
{
    constexpr int h = (T - 2) / 2;
    const double fl = floor(u);
    const int64_t st = base + (int64_t)fl - h - w_lo;
    vp = dp = vc = dc = 0.0;
    if (st < 0 || st + T > wlen) {
        atomicOr(err, ERR_WINDOW);
        return;
    }
    double w[T], dw[T];
    lagrange_wd64<T>(u - fl, w, dw);
#pragma unroll
    for (int a = 0; a < T; ++a) {
        vp = fma(w[a], sp[st + a], vp);
        dp = fma(dw[a], sp[st + a], dp);
        vc = fma(w[a], sc[st + a], vc);
        dc = fma(dw[a], sc[st + a], dc);
    }
}

template <int T>
__global__ void __launch_bounds__(256) k_sky_adj64(FwdParams P, BwdParams B)
{
    constexpr int h = (T - 2) / 2;
    extern __shared__ double sm[];
    double *hwp = sm, *hwc = sm + P.wmax;
    __shared__ TileInfo ti;
    __shared__ SkyConst skc;
    __shared__ double red[3][8];
    __shared__ double dk[2][3], du[2][3], dv[2][3];
    const int64_t total = P.total_tiles >= 0 ? P.total_tiles : P.src.tile_off[P.src.S];
    for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
        if (threadIdx.x == 0) {
            ti = tile_info(P, g, 3);
            if (!ti.ok) atomicOr(P.err, ERR_OFFSETS);
            skc = make_sky(ti.sky);
            double sl, cl, sb, cb;
            sincos(ti.sky.lam, &sl, &cl);
            sincos(ti.sky.beta, &sb, &cb);
            // derivatives of k = -e_r, u = -e_phi, v = -e_theta with respect to lambda, beta
            dk[0][0] = cb * sl;  dk[0][1] = -cb * cl; dk[0][2] = 0.0;
            dk[1][0] = sb * cl;  dk[1][1] = sb * sl;  dk[1][2] = -cb;
            du[0][0] = cl;       du[0][1] = sl;       du[0][2] = 0.0;
            du[1][0] = 0.0;      du[1][1] = 0.0;      du[1][2] = 0.0;
            dv[0][0] = sb * sl;  dv[0][1] = -sb * cl; dv[0][2] = 0.0;
            dv[1][0] = -cb * cl; dv[1][1] = -cb * sl; dv[1][2] = -sb;
        }
        __syncthreads();
        double G[3] = {0.0, 0.0, 0.0};
        if (ti.ok && ti.nb > 0) {
            const int ny = (int)ti.nb;
            const double u0 = (P.t0 - ti.t0h) / P.dt;
            const int64_t w_lo = ti.n0 + (int64_t)floor(u0) - P.sig_b - P.lproj_b - h - 2;
            const int wlen = ny + 2 * P.sig_b + P.lproj_b + T + 4;
            for (int j = threadIdx.x; j < wlen; j += blockDim.x) {
                int64_t i = w_lo + j;
                bool in = i >= 0 && i < ti.nh;
                hwp[j] = in ? __ldg(ti.hp + i) : 0.0;
                hwc[j] = in ? __ldg(ti.hc + i) : 0.0;
            }
            __syncthreads();
            const double *gy = B.g_y + 6 * (ti.out - P.out) / 3;
            for (int jj = threadIdx.x; jj < ny; jj += blockDim.x) {
                const int64_t k = ti.n0 + jj;
                double x[9], L[6];
                orbit_all(P.po, P.t0 + (double)k * P.dt, x, L);
                double sig[3];
                for (int i = 0; i < 3; ++i)
                    sig[i] = (skc.k[0] * x[3 * i] + skc.k[1] * x[3 * i + 1] + skc.k[2] * x[3 * i + 2]) / C_LIGHT *
                             P.inv_dt;
                double Rp[3], Rpd[3], Rc[3], Rcd[3];
                for (int r = 0; r < 3; ++r)
                    read_vd<T>(hwp, hwc, k, u0 - sig[r], w_lo, wlen, P.err, Rp[r], Rpd[r], Rc[r], Rcd[r]);
                for (int l = 0; l < 6; ++l) {
                    const double gl = __ldg(gy + l * ti.N + k);
                    if (gl == 0.0) continue;
                    const int LR[6] = {0, 1, 2, 0, 2, 1}, LSd[6] = {1, 2, 0, 2, 1, 0};
                    const int r = LR[l], s = LSd[l];
                    double nv[3];
                    LinkGeo q = link_geo(skc, x, l, nv);
                    double ep, epd, ec, ecd;
                    read_vd<T>(hwp, hwc, k, u0 - L[l] * P.inv_dt - sig[s], w_lo, wlen, P.err, ep, epd, ec, ecd);
                    const double dPp = ep - Rp[r], dPc = ec - Rc[r];
                    const double dH = q.xp * dPp + q.xc * dPc;
                    const double un = skc.u[0] * nv[0] + skc.u[1] * nv[1] + skc.u[2] * nv[2];
                    const double vn = skc.v[0] * nv[0] + skc.v[1] * nv[1] + skc.v[2] * nv[2];
                    for (int th = 0; th < 2; ++th) {
                        const double da = du[th][0] * nv[0] + du[th][1] * nv[1] + du[th][2] * nv[2];
                        const double db = dv[th][0] * nv[0] + dv[th][1] * nv[1] + dv[th][2] * nv[2];
                        const double dxip = 2.0 * (un * da - vn * db), dxic = 2.0 * (da * vn + un * db);
                        const double dxp = skc.c2p * dxip + skc.s2p * dxic, dxc = -skc.s2p * dxip + skc.c2p * dxic;
                        const double dkn = dk[th][0] * nv[0] + dk[th][1] * nv[1] + dk[th][2] * nv[2];
                        const double dden = 2.0 * q.den * q.den * dkn;
                        const double due = -(dk[th][0] * x[3 * s] + dk[th][1] * x[3 * s + 1] + dk[th][2] * x[3 * s + 2]) /
                                           C_LIGHT * P.inv_dt;
                        const double dur = -(dk[th][0] * x[3 * r] + dk[th][1] * x[3 * r + 1] + dk[th][2] * x[3 * r + 2]) /
                                           C_LIGHT * P.inv_dt;
                        const double ddH = dxp * dPp + dxc * dPc + q.xp * (epd * due - Rpd[r] * dur) +
                                           q.xc * (ecd * due - Rcd[r] * dur);
                        G[th] = fma(gl, dden * dH + q.den * ddH, G[th]);
                    }
                    G[2] = fma(gl, q.den * (2.0 * q.xc * dPp - 2.0 * q.xp * dPc), G[2]);
                }
            }
        }
        // fixed-order block reduction: warp tree, then warps in order
        for (int t = 0; t < 3; ++t) {
            double v = G[t];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0) red[t][threadIdx.x >> 5] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int t = 0; t < 3; ++t) {
                double s = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[t][w];
                B.partial[3 * g + t] = s;
            }
        }
        __syncthreads();
    }
}

// K4: per source, the tile partials in tile order
__global__ void k_sky_reduce(const double *partial, const int64_t *tile_off, int64_t S, int64_t ntiles1,
                             double *g_sky)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int64_t a = tile_off ? tile_off[s] : 0, b = tile_off ? tile_off[s + 1] : ntiles1;
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t t = a; t < b; ++t)
        for (int c = 0; c < 3; ++c) v[c] += partial[3 * t + c];
    for (int c = 0; c < 3; ++c) g_sky[3 * s + c] = v[c];
}

// ---------------------------------------------------------------- dispatch
#define LR_BW_ORDERS(X) X(1) X(3) X(5) X(7) X(9) X(11) X(13) X(15) X(17) X(19) X(21) X(23) X(25) X(31) X(41)

static void *bwd_kernel(int kind, int order)
{
    switch (order) {
#define LR_CASE(p)                                                                 \
    case p:                                                                        \
        return kind == 0 ? (void *)k_tdi_adj64<p + 1>                              \
                         : (kind == 1 ? (void *)k_proj_adj64<p + 1> : (void *)k_sky_adj64<p + 1>);
        LR_BW_ORDERS(LR_CASE)
#undef LR_CASE
        default: return nullptr;
    }
}

size_t smem_bwd(int kind, int order, const FwdParams &P, const BwdParams &B)
{
    const size_t T = (size_t)order + 1;
    switch (kind) {
        case 0: return sizeof(double) * (9 + T) * B.wn + sizeof(int) * B.wn;
        case 1: return sizeof(double) * (27 + T) * B.wk + sizeof(int) * B.wk;
        default: return sizeof(double) * 2 * P.wmax;
    }
}

int launch_bwd(int kind, int order, const FwdParams &P, const BwdParams &B, int sms, void *stream)
{
    void *k = bwd_kernel(kind, order);
    if (!k) return (int)cudaErrorInvalidValue;
    const size_t smem = smem_bwd(kind, order, P, B);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem);
    if (e != cudaSuccess) return (int)e;
    if (per_sm < 1) return (int)cudaErrorLaunchOutOfResources;
    int64_t grid = (int64_t)per_sm * sms;
    const int64_t known = kind == 1 ? B.h_total_tiles : P.total_tiles;
    if (known >= 0 && known < grid) grid = known;
    if (grid < 1) grid = 1;
    void *args[] = {(void *)&P, (void *)&B};
    return (int)cudaLaunchKernel(k, dim3((unsigned)grid), dim3(256), args, smem, (cudaStream_t)stream);
}

int launch_sky_reduce(const double *partial, const int64_t *tile_off, int64_t S, int64_t ntiles1, double *g_sky,
                      void *stream)
{
    const int threads = 128;
    const int64_t blocks = (S + threads - 1) / threads;
    k_sky_reduce<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(partial, tile_off, S, ntiles1, g_sky);
    return (int)cudaGetLastError();
}

}  // namespace lr
