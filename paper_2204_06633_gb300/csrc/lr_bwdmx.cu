// Mixed-precision adjoint kernels (the transposes of the TDI and projection operators for plans
// of precision LR_MIXED): float-float Lagrange weights and float-float accumulation of float-float
// cotangents on the FP32 pipe, while the orbit splines, the delays and the read positions stay FP64 and every
// index split is exact integer work on 64-bit fixed point (44 fractional bits).
//
// Structure as the FP64 kernels (lr_bwd.cu): deterministic gathers over inverted tap windows.
//   KM1  g_y = T^T g_xyz   tile of 256 link samples; per window output the six link delays in fixed
//                          point; per term float-float reference weights at the window centre with
//                          their Taylor coefficients; then per chain the chained delays by integer
//                          adds and the gather onto every link sample of the tile, each weight the
//                          reference expanded in the output's (tiny) fraction offset.
//   KM2  g_h = P^T g_y     tile of 128 strain samples; per window link sample the FP64 geometry,
//                          the 9 read positions in fixed point and the 18 coefficients as float-
//                          float, then per read the float-float weights and the gather onto every
//                          strain sample.
// Each tile's cotangents are scaled by a power of two (exactly) so that FP32 neither overflows nor
// underflows; the results are unscaled exactly.
//
//   KM3  dLoss/d(lambda, beta, psi)   tile of 256 link samples; the FP64 geometry per sample,
//                          the strain reads and their derivative reads in float-float, the assembly
//                          against g_y in FP64; per-tile partials summed in order by the FP64
//                          reduction kernel.
//
// Accuracy: the weights are float-float (~2^-45 relative), not FP32: with a static constellation
// or constant delays every read of a term has the same fraction, and FP32 weight roundings would
// act as one fixed filter error that a smooth part of the cotangent (the signal mismatch of a
// residual) sees without the cancellation of the transposed operators; the sky-angle gradient, a
// sum that cancels strongly, then moved by ~1e-6.
#include <cuda_runtime.h>

#include <climits>

#include "lr_bwd.h"
#include "lr_device.cuh"
#include "lr_mixed.cuh"
#include "lr_tdi_table.cuh"

namespace lr {
namespace {

__constant__ TdiTab c_tdibm = make_tdi_tab();
constexpr int NTERM_BW = 42;  // 3 channels x 2 chains x 7 delayed terms

// float-float reciprocals 1/d, d = 1 .. 64 (hi the FP32 rounding, lo the rounded remainder)
struct RecipTab {
    float hi[65], lo[65];
};
constexpr RecipTab make_recip_tab()
{
    RecipTab t{};
    for (int d = 1; d <= 64; ++d) {
        const double r = 1.0 / (double)d;
        t.hi[d] = (float)r;
        t.lo[d] = (float)(r - (double)(float)r);
    }
    return t;
}
__constant__ RecipTab c_recip = make_recip_tab();

// centered Lagrange weights in float-float: every factor (eps + h - a)/(a + 1) formed exactly up to
// the float-float product with the reciprocal of (a + 1); prefix products written out, then each
// multiplied by the suffix product and signed (~2^-45 relative per step)
template <int T>
__device__ __forceinline__ void lagrange_w_ff(ff e, float *whi, float *wlo, int stride)
{
    constexpr int h = (T - 2) / 2;
    ff L = {1.0f, 0.0f};
#pragma unroll 1
    for (int a = 0; a < T; ++a) {
        whi[a * stride] = L.hi;
        wlo[a * stride] = L.lo;
        L = ff_mul(L, ff_mul(ff_add_f(e, (float)(h - a)), ff{c_recip.hi[a + 1], c_recip.lo[a + 1]}));
    }
    ff R = {1.0f, 0.0f};
#pragma unroll 1
    for (int a = T - 1; a >= 0; --a) {
        const ff v = ff_mul(ff{whi[a * stride], wlo[a * stride]}, R);
        const bool neg = (T - 1 - a) & 1;
        whi[a * stride] = neg ? -v.hi : v.hi;
        wlo[a * stride] = neg ? -v.lo : v.lo;
        R = ff_mul(R, ff_mul(ff_add_f(e, (float)(h - a)), ff{c_recip.hi[T - a], c_recip.lo[T - a]}));
    }
}

__device__ __forceinline__ unsigned long long abs_bits64(double v)
{
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

// exponent se putting the largest |value| (bit pattern mb) in [1/2, 1); 0 for zero or non-finite
__device__ __forceinline__ int scale_exp(unsigned long long mb)
{
    const int eb = (int)((mb >> 52) & 0x7ffull);
    return eb >= 1 && eb <= 2044 ? 1022 - eb : 0;
}

__device__ __forceinline__ ff ff_scaled(double x, double s)
{
    const double v = x * s;  // exact (a power of two, no underflow for |x| near the tile max)
    const float hi = __double2float_rn(v);
    return {hi, __double2float_rn(v - (double)hi)};
}

// acc += (w.hi + w.lo) * (g.hi + g.lo) in float-float
__device__ __forceinline__ void ff_fma_acc2(ff &acc, float whi, float wlo, float ghi, float glo)
{
    const float p = whi * ghi;
    const float pe = fmaf(whi, ghi, -p);
    const ff s = two_sum(acc.hi, p);
    acc.hi = s.hi;
    acc.lo += s.lo + fmaf(whi, glo, fmaf(wlo, ghi, pe));
}

// ff_fma_acc2 on both lanes of packed pairs (each lane the scalar operations)
__device__ __forceinline__ void ff_fma_acc2x2(ff2 &acc, unsigned long long wh, unsigned long long wl,
                                              unsigned long long gh, unsigned long long gl)
{
    const unsigned long long p = fmul2(wh, gh);
    const unsigned long long pe = ffma2(wh, gh, fneg2(p));
    unsigned long long s, e;
    two_sum2(acc.hi, p, s, e);
    acc.hi = s;
    acc.lo = fadd2(acc.lo, fadd2(e, ffma2(wh, gl, ffma2(wl, gh, pe))));
}

__device__ __forceinline__ void block_max_u64(unsigned long long *dst, unsigned long long b)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long c = __shfl_xor_sync(0xffffffffu, b, o);
        b = c > b ? c : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(dst, b);
}

// ---------------------------------------------------------------- KM1: TDI transpose
// Every delayed read of a term at the window's outputs has a fraction within a few 1e-5 of the
// term's fraction at the window centre (the chained delays drift by ~1e-7 samples per sample), so
// its weights are the reference weights expanded to third order in the offset Delta:
//   w_a(eps_ref + Delta) = W0_a + Delta (W1_a + Delta (W2_a + Delta W3_a))
// with W0 exact in float-float and the derivatives from the product w_a = Q_a N_a: N_a the (at most
// two) factors eps / (a - h) and (eps - 1) / (a - h - 1) of the nodes next to the read, which can be
// small, differentiated exactly; Q_a the other factors (|eps + h - i| >= 1), differentiated through
// the sums S_k = sum 1 / (eps + h - i)^k (S1 in float-float); the product and the sums are formed
// once per term over all far nodes, and each tap divides its own factor out (O(T) per term instead
// of O(T) per tap).  The fourth-order term is below
// 1e-13 for |Delta| <= 5e-5.  Terms whose window crosses an integer sample (a different stencil) or
// drifts further take exact float-float weights read by read.

__device__ __forceinline__ ff recip_signed(int d)
{
    const int m = d < 0 ? -d : d;
    const ff r = {c_recip.hi[m], c_recip.lo[m]};
    return d < 0 ? ff_neg(r) : r;
}

// 1/x in float-float (~2^-46) for |x| >= 1
__device__ __forceinline__ ff recip_ff(ff x)
{
    const float r = 1.0f / x.hi;
    const float er = fmaf(-x.hi, r, 1.0f) - x.lo * r;
    return fast_two_sum(r, er * r);
}

// Constant factors of the reference weights.  With c_i = h - i (i < h) and i - h - 1 (i > h + 1),
// every factor x_i / c_i = (eps + h - i) / c_i of the far nodes lies in [1, 2) in magnitude, and
//   Q_a = prod_{i != a, h, h+1} x_i / (a - i) = P K_a / x_a   (outer taps),   P K_a   (a = h, h + 1)
// with P = prod_{i != h, h+1} x_i / c_i (one product per term) and K_a = c_a prod_{i != a, h, h+1}
// c_i / (a - i) (outer) or prod_{i != h, h+1} c_i / (a - i) (central), float-float constants.
template <int T>
struct KKTab {
    float hi[T], lo[T];
};
template <int T>
constexpr KKTab<T> make_kk_tab()
{
    KKTab<T> t{};
    constexpr int h = (T - 2) / 2;
    for (int a = 0; a < T; ++a) {
        double K = 1.0;
        for (int i = 0; i < T; ++i) {
            if (i == a || i == h || i == h + 1) continue;
            K *= (double)(i < h ? h - i : i - h - 1) / (double)(a - i);
        }
        if (a != h && a != h + 1) K *= (double)(a < h ? h - a : a - h - 1);
        t.hi[a] = (float)K;
        t.lo[a] = (float)(K - (double)(float)K);
    }
    return t;
}
template <int T>
__constant__ KKTab<T> c_kk = make_kk_tab<T>();

// per term, at its reference fraction eps: P and the sums S_k = sum_{i != h, h+1} 1 / x_i^k
// (S1 in float-float, S2 and S3 in FP32)
struct TermSums {
    ff P, S1;
    float S2, S3;
};

template <int T>
__device__ TermSums term_sums(ff e)
{
    constexpr int h = (T - 2) / 2;
    TermSums r = {{1.0f, 0.0f}, {0.0f, 0.0f}, 0.0f, 0.0f};
#pragma unroll 1
    for (int i = 0; i < T; ++i) {
        if (i == h || i == h + 1) continue;
        const ff x = ff_add_f(e, (float)(h - i));  // exact: |x| >= 1
        const int ci = i < h ? h - i : i - h - 1;
        r.P = ff_mul(r.P, ff_mul(x, ff{c_recip.hi[ci], c_recip.lo[ci]}));
        const ff rx = recip_ff(x);
        r.S1 = ff_add(r.S1, rx);
        const float r2 = rx.hi * rx.hi;
        r.S2 += r2;
        r.S3 = fmaf(r2, rx.hi, r.S3);
    }
    return r;
}

// reference weight and Taylor coefficients of tap a at eps (float-float), from the term's sums:
// the tap's own factor divided out of P and subtracted from the sums; out = W0.hi, W0.lo, W1,
// W2, W3
template <int T>
__device__ void ref_weight_taylor(ff e, int a, const TermSums &ts, float *out)
{
    constexpr int h = (T - 2) / 2;
    const ff K = {c_kk<T>.hi[a], c_kk<T>.lo[a]};
    ff Q = ff_mul(ts.P, K), S1 = ts.S1;
    float S2 = ts.S2, S3 = ts.S3;
    if (a != h && a != h + 1) {
        const ff rx = recip_ff(ff_add_f(e, (float)(h - a)));
        Q = ff_mul(Q, rx);
        S1 = ff_sub(S1, rx);
        const float r2 = rx.hi * rx.hi;
        S2 -= r2;
        S3 -= r2 * rx.hi;
    }
    ff N, N1;
    float N2 = 0.0f;
    if (a == h) {  // the factor (eps - 1) / (h - (h + 1)) = 1 - eps
        N = ff_add_f(ff_neg(e), 1.0f);
        N1 = {-1.0f, 0.0f};
    } else if (a == h + 1) {  // the factor eps / (h + 1 - h)
        N = e;
        N1 = {1.0f, 0.0f};
    } else {  // eps (eps - 1) / ((a - h)(a - h - 1))
        const ff c = ff_mul(recip_signed(a - h), recip_signed(a - h - 1));
        N = ff_mul(ff_mul(e, ff_add_f(e, -1.0f)), c);
        N1 = ff_mul(ff_add_f(ff_add(e, e), -1.0f), c);
        N2 = 2.0f * c.hi;
    }
    const ff W0 = ff_mul(Q, N);
    const ff W1 = ff_mul(Q, ff_add(ff_mul(S1, N), N1));
    const float q = Q.hi, s1 = S1.hi, n = N.hi, n1 = N1.hi;
    const float A2 = s1 * s1 - S2;
    out[0] = W0.hi;
    out[1] = W0.lo;
    out[2] = W1.hi + W1.lo;
    out[3] = 0.5f * q * (A2 * n + 2.0f * s1 * n1 + N2);
    out[4] = q * ((s1 * A2 - 2.0f * s1 * S2 + 2.0f * S3) * n + 3.0f * A2 * n1 + 3.0f * s1 * N2) * (1.0f / 6.0f);
}

// exact float-float weight of tap a at eps (the fallback)
template <int T>
__device__ __forceinline__ ff weight_ff(ff e, int a)
{
    constexpr int h = (T - 2) / 2;
    ff w = {1.0f, 0.0f};
#pragma unroll 1
    for (int i = 0; i < T; ++i)
        if (i != a) w = ff_mul(w, ff_mul(ff_add_f(e, (float)(h - i)), recip_signed(a - i)));
    return w;
}

constexpr float TAYLOR_MAX_DELTA = 5e-5f;

// Shared memory, every float array stored as (value at i, value at i + 1) pairs so that two
// consecutive taps of the gather come on the two lanes of one packed f32x2 load: RP[42][5][T]
// (W0 hi, W0 lo, W1, W2, W3 of every term and tap, as (W[a], W[a - 1])), Lf[6][WN] (int64, link
// delays in fixed point samples), Dq[WN] (int64, running chained delay of the current chain),
// Gx, Gy [3][WN] (high and low words of the scaled cotangent, as (g[j], g[j + 1])), D2[WN] (the
// offset of each output's fraction from the term's reference, as (d[j], d[j + 1])), Mo[WN] (int).
template <int T>
__global__ void __launch_bounds__(256, 2) k_tdi_adj_mx(FwdParams P, BwdParams B)
{
    constexpr int h = (T - 2) / 2;
    extern __shared__ __align__(16) long long smi[];
    const int WN = B.wn;
    float2 *RP = reinterpret_cast<float2 *>(smi);
    long long *Lf = reinterpret_cast<long long *>(RP + NTERM_BW * 5 * T), *Dq = Lf + 6 * WN;
    float2 *Gx = reinterpret_cast<float2 *>(Dq + WN), *Gy = Gx + 3 * WN, *D2 = Gy + 3 * WN;
    int *Mo = reinterpret_cast<int *>(D2 + WN);
    __shared__ TileInfo ti;
    __shared__ int mo_lo, mo_hi;
    __shared__ unsigned dmax_bits;
    __shared__ unsigned long long gmax;
    __shared__ long long dnest[NTERM_BW];
    __shared__ long long xref[NTERM_BW];  // each term's read offset at the window centre (fixed point)
    __shared__ TermSums tsum[NTERM_BW];   // each term's product and reciprocal sums at its reference
    const int64_t total = P.total_tiles >= 0 ? P.total_tiles : P.src.tile_off[P.src.S];
    for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
        if (threadIdx.x == 0) {
            ti = tile_info(P, g, 3);
            if (!ti.ok) atomicOr(P.err, ERR_OFFSETS);
            gmax = 0ull;
        }
        __syncthreads();
        if (!ti.ok || ti.nb <= 0) {
            __syncthreads();
            continue;
        }
        const int64_t N = ti.N, k0 = ti.n0, n_lo = k0 - h - 2;
        const int nb = (int)ti.nb, wn = nb + 2 * h + 5 + B.dmax;
        const int jref = wn / 2;
        const double *gx = B.g_xyz + (ti.out - P.out);
        // link delays of every window output in fixed point; the largest |g| of the window
        unsigned long long mb = 0ull;
        for (int j = threadIdx.x; j < wn; j += blockDim.x) {
            const int64_t n = n_lo + j;
            const bool in = n >= 0 && n < N;
            for (int c = 0; c < 3; ++c) mb = max(mb, in ? abs_bits64(__ldg(gx + c * N + n)) : 0ull);
            double L[6];
            orbit_delays(P.to, P.t0 + (double)n * P.dt, L);
            for (int l = 0; l < 6; ++l) Lf[l * WN + j] = __double2ll_rn(L[l] * P.inv_dt * FX_ONE);
        }
        // nested chained delays: per term the nested minus summed delay at the tile centre (it
        // changes by < 1e-10 samples over a tile), from the plan's knot table
        if (P.nest_tab && threadIdx.x < NTERM_BW) {
            const double u = (P.t0 + (double)(k0 + nb / 2) * P.dt - P.nest_t0) * P.nest_inv_dk;
            const int kk = u <= 0.0 ? 0 : (u >= (double)(P.nest_n - 2) ? P.nest_n - 2 : (int)u);
            const double f = fmin(fmax(u - (double)kk, 0.0), 1.0);
            const double a = __ldg(P.nest_tab + kk * NTERM_BW + threadIdx.x);
            const double b = __ldg(P.nest_tab + (kk + 1) * NTERM_BW + threadIdx.x);
            dnest[threadIdx.x] = llrint(fma(f, b - a, a) * FX_ONE);
        } else if (threadIdx.x < NTERM_BW) {
            dnest[threadIdx.x] = 0;
        }
        block_max_u64(&gmax, mb);
        __syncthreads();
        // each term's read offset at the window centre
        if (threadIdx.x < NTERM_BW) {
            const int id = threadIdx.x, ch = id / 14, c = (id / 7) % 2, q = id % 7 + 1;
            long long D = 0;
            for (int qq = 1; qq <= q; ++qq) D += Lf[c_tdibm.pair[ch][c][qq] * WN + jref];
            xref[id] = -(D + dnest[id]);
            const Split sr = split_fx(xref[id]);
            tsum[id] = term_sums<T>(ff{sr.ehi, sr.elo});
        }
        const int se = scale_exp(gmax);
        const double up = exp2((double)se), down = exp2((double)-se);
        for (int j = threadIdx.x; j < wn; j += blockDim.x) {
            const int64_t n = n_lo + j;
            const bool in = n >= 0 && n < N;
            for (int c = 0; c < 3; ++c) {
                const ff v = in ? ff_scaled(__ldg(gx + c * N + n), up) : ff{0.0f, 0.0f};
                Gx[c * WN + j].x = v.hi;
                Gy[c * WN + j].x = v.lo;
                if (j > 0) {
                    Gx[c * WN + j - 1].y = v.hi;
                    Gy[c * WN + j - 1].y = v.lo;
                }
                if (j == wn - 1) Gx[c * WN + j].y = Gy[c * WN + j].y = 0.0f;
            }
        }
        __syncthreads();
        // reference weights and Taylor coefficients of every (term, tap)
        for (int t = threadIdx.x; t < NTERM_BW * T; t += blockDim.x) {
            const int id = t / T, a = t - id * T;
            if (id % 7 + 1 > P.q_terms) continue;
            const Split s = split_fx(xref[id]);
            float out[5];
            ref_weight_taylor<T>(ff{s.ehi, s.elo}, a, tsum[id], out);
#pragma unroll
            for (int f = 0; f < 5; ++f) {
                float2 *row = RP + (id * 5 + f) * T;
                row[a].x = out[f];
                if (a + 1 < T) row[a + 1].y = out[f];
                if (a == 0) row[0].y = 0.0f;
            }
        }
        ff acc[6];
#pragma unroll
        for (int l = 0; l < 6; ++l) acc[l] = {0.0f, 0.0f};
        const int me = threadIdx.x;
        const int64_t k = k0 + me;
        __syncthreads();
        if (me < nb) {
            const int jk = (int)(k - n_lo);
            for (int ch = 0; ch < 3; ++ch) {
                const ff gv = {Gx[ch * WN + jk].x, Gy[ch * WN + jk].x};
#pragma unroll
                for (int l = 0; l < 6; ++l) {
                    if (l == c_tdibm.link[ch][0][0]) acc[l] = ff_add(acc[l], gv);
                    if (l == c_tdibm.link[ch][1][0]) acc[l] = ff_sub(acc[l], gv);
                }
            }
        }
        for (int ch = 0; ch < 3; ++ch)
            for (int c = 0; c < 2; ++c) {
                for (int j = threadIdx.x; j < wn; j += blockDim.x) Dq[j] = 0;
                for (int q = 1; q <= P.q_terms; ++q) {
                    const int id = (ch * 2 + c) * 7 + q - 1;
                    if (threadIdx.x == 0) {
                        mo_lo = INT_MAX;
                        mo_hi = INT_MIN;
                        dmax_bits = 0u;
                    }
                    __syncthreads();
                    const int pl = c_tdibm.pair[ch][c][q];
                    const long long xr = xref[id];
                    int lmin = INT_MAX, lmax = INT_MIN;
                    float dm = 0.0f;
                    for (int j = threadIdx.x; j < wn; j += blockDim.x) {
                        const long long D = Dq[j] + Lf[pl * WN + j];
                        Dq[j] = D;
                        const long long X = -(D + dnest[id]);  // read at n - D: index n + m
                        const int m = (int)(X >> FX_BITS);
                        Mo[j] = m;
                        lmin = min(lmin, m);
                        lmax = max(lmax, m);
                        const float d = (float)(X - xr) * 0x1p-44f;  // exact difference, then rounded
                        D2[j].x = d;
                        if (j > 0) D2[j - 1].y = d;
                        if (j == wn - 1) D2[j].y = 0.0f;
                        dm = fmaxf(dm, fabsf(d));
                    }
                    atomicMin(&mo_lo, lmin);
                    atomicMax(&mo_hi, lmax);
                    atomicMax(&dmax_bits, __float_as_uint(dm));
                    __syncthreads();
                    if (me < nb) {
                        // outputs n whose stencil [n + Mo - h, n + Mo + h + 1] contains k
                        int jlo = (int)(k - h - 1 - mo_hi - n_lo), jhi = (int)(k + h - mo_lo - n_lo);
                        jlo = max(jlo, 0);
                        jhi = min(jhi, wn - 1);
                        ff s = {0.0f, 0.0f};
                        const bool taylor = mo_lo == mo_hi && mo_lo == (int)(xr >> FX_BITS) &&
                                            __uint_as_float(dmax_bits) <= TAYLOR_MAX_DELTA;
                        if (taylor) {
                            // taps j and j + 1 (coefficient rows at a and a - 1) on the two lanes of
                            // packed pairs, two interleaved partial sums; an odd last tap alone
                            const unsigned long long *Rt =
                                reinterpret_cast<const unsigned long long *>(RP + id * 5 * T);
                            const unsigned long long *Gxc = reinterpret_cast<const unsigned long long *>(Gx + ch * WN);
                            const unsigned long long *Gyc = reinterpret_cast<const unsigned long long *>(Gy + ch * WN);
                            const unsigned long long *Dc = reinterpret_cast<const unsigned long long *>(D2);
                            int a = (int)(k - (n_lo + jlo + mo_lo)) + h;  // in [0, T): one stencil
                            ff2 S = {0ull, 0ull};
                            int j = jlo;
                            for (; j < jhi; j += 2, a -= 2) {
                                const unsigned long long d = Dc[j];
                                const unsigned long long corr =
                                    fmul2(d, ffma2(d, ffma2(d, Rt[4 * T + a], Rt[3 * T + a]), Rt[2 * T + a]));
                                ff_fma_acc2x2(S, Rt[a], fadd2(Rt[T + a], corr), Gxc[j], Gyc[j]);
                            }
                            float h0, h1, l0, l1;
                            f2unpack(S.hi, h0, h1);
                            f2unpack(S.lo, l0, l1);
                            s = ff_add(ff{h0, l0}, ff{h1, l1});
                            if (j == jhi) {
                                const float *Rs = reinterpret_cast<const float *>(RP + id * 5 * T);
                                const float d = D2[j].x;
                                const float corr = d * fmaf(d, fmaf(d, Rs[2 * (4 * T + a)], Rs[2 * (3 * T + a)]),
                                                            Rs[2 * (2 * T + a)]);
                                ff_fma_acc2(s, Rs[2 * a], Rs[2 * (T + a)] + corr, Gx[ch * WN + j].x, Gy[ch * WN + j].x);
                            }
                        } else {
                            for (int j = jlo; j <= jhi; ++j) {
                                const int a = (int)(k - (n_lo + j + Mo[j])) + h;
                                if (a >= 0 && a < T) {
                                    const long long X = -(Dq[j] + dnest[id]);
                                    const Split sp = split_fx(X);
                                    const ff w = weight_ff<T>(ff{sp.ehi, sp.elo}, a);
                                    ff_fma_acc2(s, w.hi, w.lo, Gx[ch * WN + j].x, Gy[ch * WN + j].x);
                                }
                            }
                        }
                        const int lk = c_tdibm.link[ch][c][q];
#pragma unroll
                        for (int l = 0; l < 6; ++l)
                            if (l == lk) acc[l] = c == 0 ? ff_add(acc[l], s) : ff_sub(acc[l], s);
                    }
                    __syncthreads();
                }
            }
        if (me < nb) {
            double *gy = B.g_y + 6 * (ti.out - P.out) / 3;
#pragma unroll
            for (int l = 0; l < 6; ++l) gy[l * N + k] = ((double)acc[l].hi + (double)acc[l].lo) * down;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- KM2: projection transpose
struct LinkGeoM {
    double xp, xc, den;
};

__device__ __forceinline__ LinkGeoM link_geo_m(const SkyConst &S, const double *x, int l)
{
    const int LR[6] = {0, 1, 2, 0, 2, 1}, LS[6] = {1, 2, 0, 2, 1, 0};
    const int r = LR[l], s = LS[l];
    double d0 = x[3 * r] - x[3 * s], d1 = x[3 * r + 1] - x[3 * s + 1], d2 = x[3 * r + 2] - x[3 * s + 2];
    const double inv = rsqrt(d0 * d0 + d1 * d1 + d2 * d2);
    d0 *= inv;
    d1 *= inv;
    d2 *= inv;
    const double un = S.u[0] * d0 + S.u[1] * d1 + S.u[2] * d2;
    const double vn = S.v[0] * d0 + S.v[1] * d1 + S.v[2] * d2;
    const double kn = S.k[0] * d0 + S.k[1] * d1 + S.k[2] * d2;
    const double xip = un * un - vn * vn, xic = 2.0 * un * vn;
    return {S.c2p * xip + S.s2p * xic, -S.s2p * xip + S.c2p * xic, 0.5 / (1.0 - kn)};
}

// Shared memory: X[9][WK] (int64, read positions relative to the link sample, fixed point),
// CF[18][WK] (double, then float-float pairs in place), Whi, Wlo [T][WK] (float-float weights:
// with a static constellation every sample of a read has the same fraction, as in the TDI
// transpose), Mo[WK] (int).
template <int T>
__global__ void __launch_bounds__(256, 2) k_proj_adj_mx(FwdParams P, BwdParams B)
{
    constexpr int h = (T - 2) / 2;
    extern __shared__ __align__(16) long long smi[];
    const int WK = B.wk;
    long long *X = smi;
    double *CF = reinterpret_cast<double *>(smi + 9 * WK);
    float *Whi = reinterpret_cast<float *>(smi + 27 * WK), *Wlo = Whi + T * WK;
    int *Mo = reinterpret_cast<int *>(Wlo + T * WK);
    __shared__ TileInfo ti;
    __shared__ SkyConst skc;
    __shared__ int64_t i0s, k_lo_s;
    __shared__ int nbs, wks, mo_lo, mo_hi;
    __shared__ double u0s;
    __shared__ unsigned long long cmax;
    const int64_t total = B.h_total_tiles >= 0 ? B.h_total_tiles : B.h_tile_off[P.src.S];
    for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
        if (threadIdx.x == 0) {
            FwdParams Q = P;
            Q.src.tile_off = B.h_tile_off;
            Q.tile = B.tile_h;
            ti = tile_info(Q, g, 3);
            if (!ti.ok) atomicOr(P.err, ERR_OFFSETS);
            skc = make_sky(ti.sky);
            u0s = (P.t0 - ti.t0h) / P.dt;
            cmax = 0ull;
        }
        __syncthreads();
        if (!ti.ok) {
            __syncthreads();
            continue;
        }
        if (threadIdx.x == 0) {
            // the strain tile [i0, i0 + nb) and the window of link samples whose reads reach it
            // (the same bounds as the FP64 kernel)
            const int64_t i0 = ti.n0;
            const int64_t nbh = ti.nh - i0;
            nbs = (int)(nbh < B.tile_h ? (nbh > 0 ? nbh : 0) : B.tile_h);
            i0s = i0;
            const int64_t k_ref = i0 - (int64_t)floor(u0s);
            double x[9], L[6];
            orbit_all(P.po, P.t0 + (double)k_ref * P.dt, x, L);
            double umin = 1e300, umax = -1e300;
            for (int rd = 0; rd < 9; ++rd) {
                const int sc = rd < 3 ? rd : (rd == 3 ? 1 : rd == 4 ? 2 : rd == 5 ? 0 : rd == 6 ? 2 : rd == 7 ? 1 : 0);
                double u = u0s - (skc.k[0] * x[3 * sc] + skc.k[1] * x[3 * sc + 1] + skc.k[2] * x[3 * sc + 2]) /
                                     C_LIGHT * P.inv_dt;
                if (rd >= 3) u -= L[rd - 3] * P.inv_dt;
                umin = fmin(umin, u);
                umax = fmax(umax, u);
            }
            k_lo_s = i0 - h - 2 - (int64_t)ceil(umax) - B.kmargin;
            const int64_t k_hi = i0 + nbs + h + 1 - (int64_t)floor(umin) + B.kmargin;
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
        // per window link sample: read positions (fixed point, relative to k) and coefficients
        unsigned long long mb = 0ull;
        for (int j = threadIdx.x; j < wk; j += blockDim.x) {
            const int64_t k = k_lo + j;
            if (k < 0 || k >= N) {
                for (int rd = 0; rd < 9; ++rd) {
                    X[rd * WK + j] = __double2ll_rn(u0s * FX_ONE);
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
            double rp[3] = {0.0, 0.0, 0.0}, rc[3] = {0.0, 0.0, 0.0};
            for (int l = 0; l < 6; ++l) {
                const int LR[6] = {0, 1, 2, 0, 2, 1}, LS[6] = {1, 2, 0, 2, 1, 0};
                const LinkGeoM q = link_geo_m(skc, x, l);
                const double gl = __ldg(gy + l * N + k) * q.den;
                X[(3 + l) * WK + j] = __double2ll_rn((u0s - L[l] * P.inv_dt - sig[LS[l]]) * FX_ONE);
                const double cp = gl * q.xp, cc = gl * q.xc;
                CF[(2 * (3 + l)) * WK + j] = cp;
                CF[(2 * (3 + l) + 1) * WK + j] = cc;
                mb = max(mb, max(abs_bits64(cp), abs_bits64(cc)));
                rp[LR[l]] -= cp;
                rc[LR[l]] -= cc;
            }
            for (int r = 0; r < 3; ++r) {
                X[r * WK + j] = __double2ll_rn((u0s - sig[r]) * FX_ONE);
                CF[(2 * r) * WK + j] = rp[r];
                CF[(2 * r + 1) * WK + j] = rc[r];
                mb = max(mb, max(abs_bits64(rp[r]), abs_bits64(rc[r])));
            }
        }
        block_max_u64(&cmax, mb);
        __syncthreads();
        const int se = scale_exp(cmax);
        const double up = exp2((double)se), down = exp2((double)-se);
        // coefficients to scaled float-float pairs, in place (each thread its own 8-byte slots)
        for (int t = threadIdx.x; t < 18 * wk; t += blockDim.x) {
            const int r = t / wk, j = t - r * wk;
            const ff v = ff_scaled(CF[r * WK + j], up);
            reinterpret_cast<float2 *>(CF)[r * WK + j] = make_float2(v.hi, v.lo);
        }
        __syncthreads();
        const float2 *CFf = reinterpret_cast<const float2 *>(CF);
        const int me = threadIdx.x;
        const int64_t i = i0 + me;
        ff ap = {0.0f, 0.0f}, ac = {0.0f, 0.0f};
        for (int rd = 0; rd < 9; ++rd) {
            if (threadIdx.x == 0) {
                mo_lo = INT_MAX;
                mo_hi = INT_MIN;
            }
            __syncthreads();
            int lmin = INT_MAX, lmax = INT_MIN;
            for (int j = threadIdx.x; j < wk; j += blockDim.x) {
                const Split s = split_fx(X[rd * WK + j]);
                Mo[j] = s.m;
                lmin = min(lmin, s.m);
                lmax = max(lmax, s.m);
                lagrange_w_ff<T>(ff{s.ehi, s.elo}, Whi + j, Wlo + j, WK);
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
                        const float wh = Whi[a * WK + j], wl = Wlo[a * WK + j];
                        const float2 cp = CFf[(2 * rd) * WK + j], cc = CFf[(2 * rd + 1) * WK + j];
                        ff_fma_acc2(ap, wh, wl, cp.x, cp.y);
                        ff_fma_acc2(ac, wh, wl, cc.x, cc.y);
                    }
                }
            }
            __syncthreads();
        }
        if (me < nb) {
            B.g_hp[(ti.hp - P.hp) + i] = ((double)ap.hi + (double)ap.lo) * down;
            B.g_hc[(ti.hp - P.hp) + i] = ((double)ac.hi + (double)ac.lo) * down;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- KM3: sky-angle gradient
// dLoss/d(lambda, beta, psi) = sum over link samples and links of g_y times the derivative of the
// link response (patterns, 1/(2(1 - k.n)) and the read times through k), as the FP64 kernel, with
// the strain reads and their derivative reads in float-float: value and derivative weights from
// float-float prefix and suffix products (product rule), float-float strain (scaled per tile by a
// power of two).  The geometry and the assembly against g_y stay FP64; a link and its reverse
// share the arm's unit vector (negated exactly), and the reads' power-of-two scale is undone once
// on the tile's sums.

struct LinkGeoN {
    double xp, xc, kn, den;
};

__device__ __forceinline__ LinkGeoN link_geo_n(const SkyConst &S, const double *x, int l, double *nvec)
{
    const int LR[6] = {0, 1, 2, 0, 2, 1}, LS[6] = {1, 2, 0, 2, 1, 0};
    const int r = LR[l], s = LS[l];
    double d0 = x[3 * r] - x[3 * s], d1 = x[3 * r + 1] - x[3 * s + 1], d2 = x[3 * r + 2] - x[3 * s + 2];
    const double inv = 1.0 / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    d0 *= inv;
    d1 *= inv;
    d2 *= inv;
    nvec[0] = d0;
    nvec[1] = d1;
    nvec[2] = d2;
    const double un = S.u[0] * d0 + S.u[1] * d1 + S.u[2] * d2;
    const double vn = S.v[0] * d0 + S.v[1] * d1 + S.v[2] * d2;
    LinkGeoN g;
    g.kn = S.k[0] * d0 + S.k[1] * d1 + S.k[2] * d2;
    const double xip = un * un - vn * vn, xic = 2.0 * un * vn;
    g.xp = S.c2p * xip + S.s2p * xic;
    g.xc = -S.s2p * xip + S.c2p * xic;
    g.den = 1.0 / (2.0 * (1.0 - g.kn));
    return g;
}

// value and derivative (d/dposition) of the staged float-float series at window offset st + eps:
// weights w_a = sgn L_a R_a and dw_a = sgn (L'_a R_a + L_a R'_a) from the prefix / suffix products
// and their derivatives (every factor (eps + h - i)/d linear in eps, d/deps = 1/d).  The sums are
// taken on the differences from the centre sample, s_h + sum w_a (s_a - s_h) and sum dw_a (s_a -
// s_h) (exact rewrites: the weights sum to 1, the derivative weights to 0), so the rounding scales
// with the small differences of a smooth series and not with the series itself.
template <int T>
__device__ void read_vd_ff(const float *phi, const float *plo, const float *chi, const float *clo, int st, ff e,
                           ff &vp, ff &dp, ff &vc, ff &dc)
{
    constexpr int h = (T - 2) / 2;
    ff Lp[T], Ld[T];
    ff L = {1.0f, 0.0f}, D = {0.0f, 0.0f};
#pragma unroll 1
    for (int a = 0; a < T; ++a) {
        Lp[a] = L;
        Ld[a] = D;
        const ff r = {c_recip.hi[a + 1], c_recip.lo[a + 1]};
        const ff f = ff_mul(ff_add_f(e, (float)(h - a)), r);
        D = ff_add(ff_mul(D, f), ff_mul(L, r));
        L = ff_mul(L, f);
    }
    const ff cp = {phi[st + h], plo[st + h]}, cc = {chi[st + h], clo[st + h]};
    // h+ and hx on the two lanes of packed pairs (each lane the scalar float-float operations)
    const ff2 C2 = {f2pack(cp.hi, cc.hi), f2pack(cp.lo, cc.lo)};
    ff2 V = {0ull, 0ull}, DV = {0ull, 0ull};
    ff R = {1.0f, 0.0f}, RD = {0.0f, 0.0f};
#pragma unroll 1
    for (int a = T - 1; a >= 0; --a) {
        ff w = ff_mul(Lp[a], R), dw = ff_add(ff_mul(Ld[a], R), ff_mul(Lp[a], RD));
        if ((T - 1 - a) & 1) {
            w = ff_neg(w);
            dw = ff_neg(dw);
        }
        const ff2 S = ff_sub2(ff2{f2pack(phi[st + a], chi[st + a]), f2pack(plo[st + a], clo[st + a])}, C2);
        ff_fma_acc2x2(V, f2pack(w.hi, w.hi), f2pack(w.lo, w.lo), S.hi, S.lo);
        ff_fma_acc2x2(DV, f2pack(dw.hi, dw.hi), f2pack(dw.lo, dw.lo), S.hi, S.lo);
        const ff r = {c_recip.hi[T - a], c_recip.lo[T - a]};
        const ff g = ff_mul(ff_add_f(e, (float)(h - a)), r);
        RD = ff_add(ff_mul(RD, g), ff_mul(R, r));
        R = ff_mul(R, g);
    }
    f2unpack(V.hi, vp.hi, vc.hi);
    f2unpack(V.lo, vp.lo, vc.lo);
    f2unpack(DV.hi, dp.hi, dc.hi);
    f2unpack(DV.lo, dp.lo, dc.lo);
    vp = ff_add(vp, cp);
    vc = ff_add(vc, cc);
}

// reads at window offset base + u (FP64 position): index split in FP64, fraction as float-float;
// results unscaled to FP64.  An out-of-window stencil records ERR_WINDOW and reads 0.
template <int T>
__device__ __forceinline__ void read_vd_mx(const float *sm, int wstride, int64_t base, double u, int64_t w_lo,
                                           int wlen, double down, int *err, double &vp, double &dp, double &vc,
                                           double &dc)
{
    constexpr int h = (T - 2) / 2;
    const double fl = floor(u);
    const int64_t st = base + (int64_t)fl - h - w_lo;
    vp = dp = vc = dc = 0.0;
    if (st < 0 || st + T > wlen) {
        atomicOr(err, ERR_WINDOW);
        return;
    }
    const double ed = u - fl;
    const float eh = __double2float_rn(ed);
    ff a, b, c, d;
    read_vd_ff<T>(sm, sm + wstride, sm + 2 * wstride, sm + 3 * wstride, (int)st, ff{eh, __double2float_rn(ed - eh)}, a,
                  b, c, d);
    vp = ((double)a.hi + (double)a.lo) * down;
    dp = ((double)b.hi + (double)b.lo) * down;
    vc = ((double)c.hi + (double)c.lo) * down;
    dc = ((double)d.hi + (double)d.lo) * down;
}

template <int T>
__global__ void __launch_bounds__(256, 2) k_sky_adj_mx(FwdParams P, BwdParams B)
{
    constexpr int h = (T - 2) / 2;
    extern __shared__ __align__(16) float sms[];  // h+ hi, h+ lo, hx hi, hx lo: [4][wmax]
    const int WS = P.wmax;
    __shared__ TileInfo ti;
    __shared__ SkyConst skc;
    __shared__ double red[3][8];
    __shared__ double dk[2][3], du[2][3], dv[2][3];
    __shared__ unsigned long long hmax;
    const int64_t total = P.total_tiles >= 0 ? P.total_tiles : P.src.tile_off[P.src.S];
    for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
        if (threadIdx.x == 0) {
            ti = tile_info(P, g, 3);
            if (!ti.ok) atomicOr(P.err, ERR_OFFSETS);
            skc = make_sky(ti.sky);
            hmax = 0ull;
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
            unsigned long long mb = 0ull;
            for (int j = threadIdx.x; j < wlen; j += blockDim.x) {
                const int64_t i = w_lo + j;
                const bool in = i >= 0 && i < ti.nh;
                mb = max(mb, in ? max(abs_bits64(__ldg(ti.hp + i)), abs_bits64(__ldg(ti.hc + i))) : 0ull);
            }
            block_max_u64(&hmax, mb);
            __syncthreads();
            const int se = scale_exp(hmax);
            const double up = exp2((double)se), down = exp2((double)-se);
            for (int j = threadIdx.x; j < wlen; j += blockDim.x) {
                const int64_t i = w_lo + j;
                const bool in = i >= 0 && i < ti.nh;
                const ff a = in ? ff_scaled(__ldg(ti.hp + i), up) : ff{0.0f, 0.0f};
                const ff b = in ? ff_scaled(__ldg(ti.hc + i), up) : ff{0.0f, 0.0f};
                sms[j] = a.hi;
                sms[WS + j] = a.lo;
                sms[2 * WS + j] = b.hi;
                sms[3 * WS + j] = b.lo;
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
                // reads still scaled by the tile's power of two: every term below is linear in them,
                // so the sums are unscaled once at the end of the tile
                double Rp[3], Rpd[3], Rc[3], Rcd[3];
                for (int r = 0; r < 3; ++r)
                    read_vd_mx<T>(sms, WS, k, u0 - sig[r], w_lo, wlen, 1.0, P.err, Rp[r], Rpd[r], Rc[r], Rcd[r]);
                // arm a carries link a (receiver a, emitter a + 1) and its reverse 5 - a: the reverse
                // has the unit vector negated exactly, so the patterns and their angle derivatives are
                // the same and k.n and its derivatives change sign
                for (int arm = 0; arm < 3; ++arm) {
                    const double g0 = __ldg(gy + arm * ti.N + k), g1 = __ldg(gy + (5 - arm) * ti.N + k);
                    if (g0 == 0.0 && g1 == 0.0) continue;
                    double nv[3];
                    const LinkGeoN q = link_geo_n(skc, x, arm, nv);
                    const double un = skc.u[0] * nv[0] + skc.u[1] * nv[1] + skc.u[2] * nv[2];
                    const double vn = skc.v[0] * nv[0] + skc.v[1] * nv[1] + skc.v[2] * nv[2];
                    double dxp[2], dxc[2], dkn[2];
                    for (int th = 0; th < 2; ++th) {
                        const double da = du[th][0] * nv[0] + du[th][1] * nv[1] + du[th][2] * nv[2];
                        const double db = dv[th][0] * nv[0] + dv[th][1] * nv[1] + dv[th][2] * nv[2];
                        const double dxip = 2.0 * (un * da - vn * db), dxic = 2.0 * (da * vn + un * db);
                        dxp[th] = skc.c2p * dxip + skc.s2p * dxic;
                        dxc[th] = -skc.s2p * dxip + skc.c2p * dxic;
                        dkn[th] = dk[th][0] * nv[0] + dk[th][1] * nv[1] + dk[th][2] * nv[2];
                    }
                    for (int rev = 0; rev < 2; ++rev) {
                        const double gl = rev ? g1 : g0;
                        if (gl == 0.0) continue;
                        const int l = rev ? 5 - arm : arm;
                        const int LR[6] = {0, 1, 2, 0, 2, 1}, LS[6] = {1, 2, 0, 2, 1, 0};
                        const int r = LR[l], s = LS[l];
                        const double sg = rev ? -1.0 : 1.0;
                        const double den = rev ? 1.0 / (2.0 * (1.0 + q.kn)) : q.den;
                        double ep, epd, ec, ecd;
                        read_vd_mx<T>(sms, WS, k, u0 - L[l] * P.inv_dt - sig[s], w_lo, wlen, 1.0, P.err, ep, epd, ec,
                                      ecd);
                        const double dPp = ep - Rp[r], dPc = ec - Rc[r];
                        const double dH = q.xp * dPp + q.xc * dPc;
                        for (int th = 0; th < 2; ++th) {
                            const double dden = 2.0 * den * den * (sg * dkn[th]);
                            const double due = -(dk[th][0] * x[3 * s] + dk[th][1] * x[3 * s + 1] + dk[th][2] * x[3 * s + 2]) /
                                               C_LIGHT * P.inv_dt;
                            const double dur = -(dk[th][0] * x[3 * r] + dk[th][1] * x[3 * r + 1] + dk[th][2] * x[3 * r + 2]) /
                                               C_LIGHT * P.inv_dt;
                            const double ddH = dxp[th] * dPp + dxc[th] * dPc + q.xp * (epd * due - Rpd[r] * dur) +
                                               q.xc * (ecd * due - Rcd[r] * dur);
                            G[th] = fma(gl, dden * dH + den * ddH, G[th]);
                        }
                        G[2] = fma(gl, den * (2.0 * q.xc * dPp - 2.0 * q.xp * dPc), G[2]);
                    }
                }
            }
            for (int t = 0; t < 3; ++t) G[t] *= down;
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
                double acc = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) acc += red[t][w];
                B.partial[3 * g + t] = acc;
            }
        }
        __syncthreads();
    }
}

#define LR_BM_ORDERS(X) X(1) X(3) X(5) X(7) X(9) X(11) X(13) X(15) X(17) X(19) X(21) X(23) X(25) X(31) X(41)

void *bwd_kernel_mx(int kind, int order)
{
    switch (order) {
#define LR_CASE(p) \
    case p: return kind == 0 ? (void *)k_tdi_adj_mx<p + 1> : kind == 1 ? (void *)k_proj_adj_mx<p + 1> \
                                                                        : (void *)k_sky_adj_mx<p + 1>;
        LR_BM_ORDERS(LR_CASE)
#undef LR_CASE
        default: return nullptr;
    }
}

}  // namespace

size_t smem_bwd_mx(int kind, int order, const FwdParams &P, const BwdParams &B)
{
    const size_t T = (size_t)order + 1;
    if (kind == 2) return sizeof(float) * 4 * (size_t)P.wmax;
    return kind == 0 ? (size_t)B.wn * (7 * 8 + 6 * 8 + 8 + 4) + (size_t)NTERM_BW * 5 * T * 8
                     : (size_t)B.wk * (27 * 8 + 2 * T * 4 + 4);
}

int launch_bwd_mx(int kind, int order, const FwdParams &P, const BwdParams &B, int sms, void *stream)
{
    void *k = bwd_kernel_mx(kind, order);
    if (!k) return (int)cudaErrorInvalidValue;
    const size_t smem = smem_bwd_mx(kind, order, P, B);
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

}  // namespace lr
