// Building blocks of the mixed-precision response: float-float arithmetic, exact fixed-point
// index splits, and the compensated Lagrange read (FP32 taps on third differences).
//
// Why compensated: the link response is a difference of two nearly equal strain reads
// (|y|/|h| ~ 2 pi f L) and TDI-2 cancels the link series again by ~8 (2 pi f L)^2, so at
// 0.1 mHz the output is ~1e-6 of the strain.  Plain FP32 taps and data then carry relative
// errors of order one.  Here every read is split exactly as
//     P(eps) = [s_m + eps d_m]                                   float-float
//            + eps (eps - 1) a_m  -  sum_a U_a(eps) e_{m-h+a}        FP32
// with d = first difference, a = half second difference, e = third difference of the
// series (all formed from the float-float values), and U the triple running sums of the
// Lagrange weights minus the quadratic Newton weights on the nodes -1, 0, 1 (which vanish
// on quadratics, so the sum of their products with the data equals minus the sum of U with
// the third differences, by three summations by parts).  The FP32 part only ever
// multiplies small, smooth quantities.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lr {

// ---------------------------------------------------------------- float-float
// A value hi + lo with |lo| <= ulp(hi)/2 (about 48 significant bits).  Error-free
// transformations: two_sum (Knuth, TAOCP vol. 2, 4.2.2) and two_prod via fused multiply-add.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b)
{
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b)
{
    float s = a + b;
    float e = b - (s - a);
    return {s, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    ff s = two_sum(a.hi, b.hi);
    float lo = s.lo + (a.lo + b.lo);
    return fast_two_sum(s.hi, lo);
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_add_f(ff a, float b)
{
    ff s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, s.lo + a.lo);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b)
{
    float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_from_double(double x)
{
    float h = __double2float_rn(x);
    float l = __double2float_rn(x - (double)h);
    return {h, l};
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// ---------------------------------------------------------------- fixed-point index split
// Positions and delays in samples are carried as 64-bit fixed point with 44 fractional bits
// (resolution 5.7e-14 sample), converted once from the FP64 spline evaluation; the split into
// the integer index m = floor(x) and the fraction eps = x - m is then exact integer work:
// eps is returned as hi + lo with hi holding the top 23 fraction bits and lo the next 21.
constexpr int FX_BITS = 44;
constexpr double FX_ONE = 17592186044416.0;  // 2^44

struct Split {
    int m;
    float ehi, elo;
};

__device__ __forceinline__ Split split_fx(long long X)
{
    Split s;
    s.m = (int)(X >> FX_BITS);
    unsigned long long f = (unsigned long long)X & ((1ull << FX_BITS) - 1ull);
    unsigned top = (unsigned)(f >> 21);
    unsigned bot = (unsigned)(f & ((1u << 21) - 1u));
    s.ehi = __int_as_float(0x3F800000u | top) - 1.0f;
    s.elo = (__int_as_float(0x3F800000u | (bot << 2)) - 1.0f) * 0x1p-23f;
    return s;
}

// ---------------------------------------------------------------- compensated weights
// U[0 .. T-4]: triple running sums of r = w - q, where w are the degree-(T-1) centered
// Lagrange weights at eps (nodes a - h, h = (T-2)/2) and q the quadratic weights on the
// nodes -1, 0, 1 (a = h-1, h, h+1).  Left of the centre the sums run from the left end;
// from the centre on they run from the right end (r has three vanishing moments, so both
// give the same U), which keeps each sum short and its rounding small.
template <int T>
__device__ __forceinline__ void comp_weights(float e, float *U)
{
    constexpr int h = (T - 2) / 2;
    float w[T];
    // prefix products L_a = prod_{i<a} (e + h - i)/(i + 1), then w_a = sgn L_a R_a with the
    // suffix products R_a = prod_{i>a} (e + h - i)/(T - i) accumulated from the right
    float L = 1.0f;
#pragma unroll
    for (int a = 0; a < T; ++a) {
        w[a] = L;
        L = L * fmaf(e, 1.0f / (float)(a + 1), (float)(h - a) / (float)(a + 1));
    }
    float R = 1.0f;
#pragma unroll
    for (int a = T - 1; a >= 0; --a) {
        const float sg = ((T - 1 - a) & 1) ? -1.0f : 1.0f;
        w[a] = sg * w[a] * R;
        R = R * fmaf(e, 1.0f / (float)(T - a), (float)(h - a) / (float)(T - a));
    }
    const float em1 = e - 1.0f;
    w[h - 1] -= 0.5f * e * em1;
    w[h] -= (1.0f - e) * (1.0f + e);
    w[h + 1] -= 0.5f * e * (e + 1.0f);
    // left: forward sums over a = 0 .. h-1
    float s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll
    for (int a = 0; a < h; ++a) {
        s1 += w[a];
        s2 += s1;
        s3 += s2;
        if (a <= T - 4) U[a] = s3;
    }
    // right: U1_a = -sum_{b>a} r_b, U2_a = -sum_{a<b<=T-2} U1_b, U3_a = -sum_{a<b<=T-3} U2_b
    float t1 = 0.0f, t2 = 0.0f, t3 = 0.0f;
    float u1[T], u2[T];
#pragma unroll
    for (int a = T - 2; a >= h; --a) {
        t1 -= w[a + 1];
        u1[a] = t1;
    }
#pragma unroll
    for (int a = T - 3; a >= h; --a) {
        t2 -= u1[a + 1];
        u2[a] = t2;
    }
#pragma unroll
    for (int a = T - 4; a >= h; --a) {
        t3 -= u2[a + 1];
        U[a] = t3;
    }
}

// Staged series in shared memory for compensated reads: value s (float-float), first
// difference d = s_{j+1} - s_j (float-float), a = (s_{j+1} - 2 s_j + s_{j-1})/2 (FP32, plus its
// low part alo for the strain, whose curvature term feeds two levels of cancellation) and
// e = s_{j+3} - 3 s_{j+2} + 3 s_{j+1} - s_j (FP32).
struct CompSeries {
    float *shi, *slo, *dhi, *dlo, *a, *e, *alo;
};

// float-float s_m + eps d_m + eps (eps - 1) a_m - C; with FFQ the curvature product is formed
// exactly (two_prod of eps_hi (eps_hi - 1), whose factors are exact in FP32) against the
// float-float a_m, otherwise in FP32
template <bool FFQ>
__device__ __forceinline__ ff comp_finish(const CompSeries &S, int m, float ehi, float elo, float C)
{
    ff d = {S.dhi[m], S.dlo[m]};
    float p = ehi * d.hi;
    float pe = fmaf(ehi, d.hi, -p);
    pe = fmaf(ehi, d.lo, pe);
    pe = fmaf(elo, d.hi, pe);
    ff r = ff_add({S.shi[m], S.slo[m]}, fast_two_sum(p, pe));
    if constexpr (FFQ) {
        const float em1 = ehi - 1.0f;
        float q = ehi * em1;
        float qe = fmaf(ehi, em1, -q);
        qe = fmaf(elo, 2.0f * ehi - 1.0f, qe);
        ff cq = ff_mul(fast_two_sum(q, qe), {S.a[m], S.alo[m]});
        r = ff_add(r, cq);
        r = ff_add_f(r, -C);
    } else {
        float small = fmaf(ehi * (ehi - 1.0f), S.a[m], -C);
        r = ff_add_f(r, small);
    }
    return r;
}

// One compensated read at window index m (the anchor node) with fraction eps = ehi + elo
// and correction weights U; returns the float-float value of the interpolant.
template <int T, bool FFQ = false>
__device__ __forceinline__ ff comp_value(const CompSeries &S, int m, float ehi, float elo, const float *U)
{
    constexpr int h = (T - 2) / 2;
    float C = 0.0f;
    if constexpr (T >= 4) {
        const float *ep = S.e + (m - h);
#pragma unroll
        for (int a = 0; a <= T - 4; ++a) C = fmaf(U[a], ep[a], C);
        return comp_finish<FFQ>(S, m, ehi, elo, C);
    } else {
        // degree 1: the interpolant is the linear anchor itself
        ff d = {S.dhi[m], S.dlo[m]};
        float p = ehi * d.hi;
        float pe = fmaf(ehi, d.hi, -p);
        pe = fmaf(ehi, d.lo, pe);
        pe = fmaf(elo, d.hi, pe);
        return ff_add({S.shi[m], S.slo[m]}, fast_two_sum(p, pe));
    }
}

// The same read with the correction sum taken from a first-order expansion of U around a
// reference fraction (U0 + delta U1); the anchor and the curvature term use the exact eps.
template <int T>
__device__ __forceinline__ ff comp_value_taylor(const CompSeries &S, int m, float ehi, float elo, const float *U0,
                                                const float *U1, float delta)
{
    constexpr int h = (T - 2) / 2;
    if constexpr (T >= 4) {
        float C = 0.0f, C1 = 0.0f;
        const float *ep = S.e + (m - h);
#pragma unroll
        for (int a = 0; a <= T - 4; ++a) {
            float v = ep[a];
            C = fmaf(U0[a], v, C);
            C1 = fmaf(U1[a], v, C1);
        }
        C = fmaf(delta, C1, C);
        return comp_finish<false>(S, m, ehi, elo, C);
    } else {
        return comp_value<T>(S, m, ehi, elo, U0);
    }
}

}  // namespace lr
