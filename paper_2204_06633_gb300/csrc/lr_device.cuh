// Device building blocks shared by the response kernels: orbit splines, sky frame, tile
// bookkeeping and the centered Lagrange fractional-delay read.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lr_gb.cuh"
#include "lr_internal.h"

namespace lr {

// ---------------------------------------------------------------- splines
struct alignas(32) Coef4 {
    double a, b, c, d;
};

__device__ inline const Coef4 *spline_row(const OrbitDev &o, double t, double *x)
{
    double u = (t - o.t_first) * o.inv_dk;
    double fl = floor(u);
    int k = (int)fl;
    k = k < 0 ? 0 : (k > o.nint - 1 ? o.nint - 1 : k);
    *x = u - (double)k;
    return reinterpret_cast<const Coef4 *>(o.coef) + (size_t)k * NSERIES;
}

__device__ inline Coef4 ldg4(const Coef4 *p)
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 u = __ldg(q), v = __ldg(q + 1);
    Coef4 r;
    r.a = u.x; r.b = u.y; r.c = v.x; r.d = v.y;
    return r;
}

__device__ inline double cubic(const Coef4 &q, double x) { return fma(x, fma(x, fma(x, q.d, q.c), q.b), q.a); }

// positions [9] and delays [6] at t
__device__ inline void orbit_all(const OrbitDev &o, double t, double *pos, double *del)
{
    double x;
    const Coef4 *row = spline_row(o, t, &x);
#pragma unroll
    for (int s = 0; s < 9; ++s) pos[s] = cubic(ldg4(row + s), x);
#pragma unroll
    for (int l = 0; l < 6; ++l) del[l] = cubic(ldg4(row + 9 + l), x);
}

__device__ inline void orbit_delays(const OrbitDev &o, double t, double *del)
{
    double x;
    const Coef4 *row = spline_row(o, t, &x);
#pragma unroll
    for (int l = 0; l < 6; ++l) del[l] = cubic(ldg4(row + 9 + l), x);
}

__device__ inline double orbit_delay1(const OrbitDev &o, double t, int l)
{
    double x;
    const Coef4 *row = spline_row(o, t, &x);
    return cubic(ldg4(row + 9 + l), x);
}

// ---------------------------------------------------------------- tiles
struct TileInfo {
    int64_t n0, nb, N, nh;
    double t0h;
    lr_sky sky;
    const double *hp, *hc;
    double *out;      // base of this source's output block
    const double *yin;
    const double *dat;  // base of this source's A, E, T data (likelihood launches), else null
    GbConst gb;         // generated strain: the source's Galactic-binary constants
    int ok;
};

// Maps global tile g to its source.  `ochan` is the number of output channels (3 for TDI,
// 6 for link series).
// A, E, T data block of the source with outputs [oo, oo1): null (and ERR_OFFSETS) when the
// offsets run past the data the caller declared
__device__ inline const double *like_data(const FwdParams &P, int64_t oo, int64_t oo1)
{
    if (!P.like.data) return nullptr;
    if (oo < 0 || oo1 < oo || oo1 > P.like.n_total) {
        atomicOr(P.err, ERR_OFFSETS);
        return nullptr;
    }
    return P.like.data + 3 * oo;
}

__device__ inline TileInfo tile_info(const FwdParams &P, int64_t g, int ochan)
{
    TileInfo ti;
    ti.ok = 1;
    if (P.src.tile_off == nullptr) {
        ti.N = P.src.n1;
        ti.nh = P.src.nh1;
        ti.t0h = P.src.t0h1;
        ti.sky = P.src.sky1;
        ti.hp = P.hp;
        ti.hc = P.hc;
        ti.out = P.out;
        ti.yin = P.yin;
        ti.dat = P.like.data;
        ti.n0 = g * P.tile;
        if (P.gen_strain) ti.gb = make_gb(P.src.gb1);
    } else {
        const int64_t *to = P.src.tile_off;
        int64_t lo = 0, hi = P.src.S;  // find s with to[s] <= g < to[s+1]
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) >> 1;
            if (__ldg(to + mid) <= g) lo = mid; else hi = mid;
        }
        int64_t s = lo;
        int64_t ho = 0, ho1 = 0;
        if (P.gen_strain) {
            ti.gb = make_gb(P.src.gb[s]);
        } else {
            ho = __ldg(P.src.h_off + s);
            ho1 = __ldg(P.src.h_off + s + 1);
        }
        int64_t oo = __ldg(P.src.out_off + s), oo1 = __ldg(P.src.out_off + s + 1);
        ti.N = oo1 - oo;
        ti.nh = ho1 - ho;
        if (ti.N < 0 || ti.nh < 0) ti.ok = 0;
        ti.t0h = P.gen_strain ? P.t0 : __ldg(P.src.t0h + s);
        ti.sky = P.src.sky[s];
        ti.hp = P.hp + ho;
        ti.hc = P.hc + ho;
        ti.out = P.out ? P.out + ochan * oo : nullptr;
        ti.yin = P.yin ? P.yin + 6 * oo : nullptr;
        ti.dat = like_data(P, oo, oo1);
        ti.n0 = (g - __ldg(to + s)) * P.tile;
    }
    if (P.gen_strain) {
        ti.nh = GEN_STRAIN_LEN;
        ti.t0h = P.t0;
    }
    int64_t rem = ti.N - ti.n0;
    ti.nb = rem < P.tile ? rem : P.tile;
    if (ti.nb < 0) ti.nb = 0;
    return ti;
}

// ---------------------------------------------------------------- Lagrange reads (FP64)
// Centered Lagrange interpolation of degree p = T-1 through the nodes j = -h .. h+1
// (h = (p-1)/2) at offset eps, w_a = (-1)^(T-1-a) L_a R_a with the prefix products
// L_a = prod_{i<a} (eps+h-i)/(i+1) and suffix products R_a = prod_{i>a} (eps+h-i)/(T-i).
// The sum  sum_a w_a s_a  is evaluated in nested (Horner) form over the suffix factors
// f_a = (eps+h-a)/(T-a):  acc_a = acc_{a-1} f_a + sgn L_a s_a,  so no weight array is kept.
template <int T>
__device__ __forceinline__ double horner1(const double *__restrict__ s, double e)
{
    constexpr int h = (T - 2) / 2;
    double L = -1.0;
    double acc = -s[0];
#pragma unroll
    for (int j = 1; j < T; ++j) {
        const double cf1 = 1.0 / (double)(T - j), cf0 = (double)(h - j) / (double)(T - j);
        const double cg1 = -1.0 / (double)j, cg0 = (double)(j - 1 - h) / (double)j;
        double f = fma(e, cf1, cf0);
        L = L * fma(e, cg1, cg0);
        acc = fma(acc, f, L * s[j]);
    }
    return acc;
}

template <int T>
__device__ __forceinline__ void horner2(const double *__restrict__ a, const double *__restrict__ b, double e,
                                        double &ra, double &rb)
{
    constexpr int h = (T - 2) / 2;
    double L = -1.0;
    double acca = -a[0], accb = -b[0];
#pragma unroll
    for (int j = 1; j < T; ++j) {
        const double cf1 = 1.0 / (double)(T - j), cf0 = (double)(h - j) / (double)(T - j);
        const double cg1 = -1.0 / (double)j, cg0 = (double)(j - 1 - h) / (double)j;
        double f = fma(e, cf1, cf0);
        L = L * fma(e, cg1, cg0);
        acca = fma(acca, f, L * a[j]);
        accb = fma(accb, f, L * b[j]);
    }
    ra = acca;
    rb = accb;
}

// Reads series staged in shared memory at sample position base + u, where the staged
// window starts at absolute index w_lo and holds wlen samples.  A stencil outside the
// window records ERR_WINDOW and reads as 0 (never touches memory outside the window).
template <int T>
__device__ __forceinline__ double read1(const double *s, int64_t base, double u, int64_t w_lo, int wlen, int *err)
{
    constexpr int h = (T - 2) / 2;
    double fl = floor(u);
    double e = u - fl;
    int64_t st = base + (int64_t)fl - h - w_lo;
    if (st < 0 || st + T > wlen) {
        atomicOr(err, ERR_WINDOW);
        return 0.0;
    }
    return horner1<T>(s + st, e);
}

template <int T>
__device__ __forceinline__ void read2(const double *a, const double *b, int64_t base, double u, int64_t w_lo,
                                      int wlen, double &ra, double &rb, int *err)
{
    constexpr int h = (T - 2) / 2;
    double fl = floor(u);
    double e = u - fl;
    int64_t st = base + (int64_t)fl - h - w_lo;
    if (st < 0 || st + T > wlen) {
        atomicOr(err, ERR_WINDOW);
        ra = rb = 0.0;
        return;
    }
    horner2<T>(a + st, b + st, e, ra, rb);
}


// ---------------------------------------------------------------- likelihood epilogue
// Adds the terms of one output sample (X, Y, Z of the template; dA, dE, dT of the data) to the
// partial inner products <d|h> and <h|h> over the channels A = (Z - X)/sqrt 2,
// E = (X - 2 Y + Z)/sqrt 6, T = (X + Y + Z)/sqrt 3 with weights w.
__device__ inline void like_terms(const LikeArgs &L, double X, double Y, double Z, double dA, double dE, double dT,
                                  double &dh, double &hh)
{
    const double R2 = 0.70710678118654752440, R6 = 0.40824829046386301637, R3 = 0.57735026918962576451;
    const double s = X + Z;
    const double a = (Z - X) * R2, e = fma(-2.0, Y, s) * R6, t = (s + Y) * R3;
    const double wa = L.w[0] * a, we = L.w[1] * e, wt = L.w[2] * t;
    dh = fma(wa, dA, fma(we, dE, fma(wt, dT, dh)));
    hh = fma(wa, a, fma(we, e, fma(wt, t, hh)));
}

// Block sum of (a, b) in a fixed order (shuffle tree within warps, then warps in index order);
// red holds 2 doubles per warp.  Every thread of the block must call it; thread 0 gets the sums.
__device__ inline void block_sum2(double &a, double &b, double *red)
{
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[2 * w] = a;
        red[2 * w + 1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int i = 0; i < nw; ++i) {
            sa += red[2 * i];
            sb += red[2 * i + 1];
        }
        a = sa;
        b = sb;
    }
}

__device__ inline double nan_d() { return __longlong_as_double(0x7ff8000000000000ll); }

// tile g's partial, or ERR_OFFSETS when g is past the partial buffer
__device__ inline void like_store(const FwdParams &P, int64_t g, double dh, double hh)
{
    if (g < 0 || g >= P.like.cap) {
        atomicOr(P.err, ERR_OFFSETS);
        return;
    }
    P.like.partial[2 * g] = dh;
    P.like.partial[2 * g + 1] = hh;
}

}  // namespace lr
