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
// U[a] from r = w - q: left of the centre the triple running sums run from the left end; from
// the centre on they run from the right end (r has three vanishing moments, so both give the
// same U), which keeps each sum short and its rounding small.
template <int T>
__device__ __forceinline__ void triple_sums(const float *r, float *U)
{
    constexpr int h = (T - 2) / 2;
    float s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll
    for (int a = 0; a < h; ++a) {
        s1 += r[a];
        s2 += s1;
        s3 += s2;
        if (a <= T - 4) U[a] = s3;
    }
    // right: U1_a = -sum_{b>a} r_b, U2_a = -sum_{a<b<=T-2} U1_b, U3_a = -sum_{a<b<=T-3} U2_b
    float t1 = 0.0f, t2 = 0.0f, t3 = 0.0f;
    float u1[T], u2[T];
#pragma unroll
    for (int a = T - 2; a >= h; --a) {
        t1 -= r[a + 1];
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

// U[0 .. T-4]: triple running sums of r = w - q, where w are the degree-(T-1) centered
// Lagrange weights at eps (nodes a - h, h = (T-2)/2) and q the quadratic weights on the
// nodes -1, 0, 1 (a = h-1, h, h+1).
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
    triple_sums<T>(w, U);
}

// U and its exact derivative dU/deps at eps: the product rule carried through the prefix and
// suffix products (each factor is linear in eps), the derivatives of the quadratic weights
// subtracted, and the same triple sums applied to both (they are linear).
template <int T>
__device__ __forceinline__ void comp_weights_d(float e, float *U, float *U1)
{
    constexpr int h = (T - 2) / 2;
    float w[T], wd[T];
    float L = 1.0f, Ld = 0.0f;
#pragma unroll
    for (int a = 0; a < T; ++a) {
        w[a] = L;
        wd[a] = Ld;
        const float c1 = 1.0f / (float)(a + 1), c0 = (float)(h - a) / (float)(a + 1);
        const float f = fmaf(e, c1, c0);
        Ld = fmaf(Ld, f, L * c1);
        L = L * f;
    }
    float R = 1.0f, Rd = 0.0f;
#pragma unroll
    for (int a = T - 1; a >= 0; --a) {
        const float sg = ((T - 1 - a) & 1) ? -1.0f : 1.0f;
        wd[a] = sg * fmaf(wd[a], R, w[a] * Rd);
        w[a] = sg * w[a] * R;
        const float c1 = 1.0f / (float)(T - a), c0 = (float)(h - a) / (float)(T - a);
        const float g = fmaf(e, c1, c0);
        Rd = fmaf(Rd, g, R * c1);
        R = R * g;
    }
    w[h - 1] -= 0.5f * e * (e - 1.0f);
    w[h] -= (1.0f - e) * (1.0f + e);
    w[h + 1] -= 0.5f * e * (e + 1.0f);
    wd[h - 1] -= e - 0.5f;
    wd[h] += 2.0f * e;
    wd[h + 1] -= e + 0.5f;
    triple_sums<T>(w, U);
    triple_sums<T>(wd, U1);
}

// ---------------------------------------------------------------- packed f32x2 pairs
// packed pairs of FP32 values and their fused multiply-add (fma.rn.f32x2: two IEEE FMAs in one
// instruction)
__device__ __forceinline__ unsigned long long f2pack(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ void f2unpack(unsigned long long r, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}

__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ unsigned long long fadd2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ unsigned long long fsub2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ unsigned long long fmul2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// both lanes negated (sign bits flipped)
__device__ __forceinline__ unsigned long long fneg2(unsigned long long a) { return a ^ 0x8000000080000000ull; }

// two_sum on both lanes of packed pairs (each lane exactly the scalar two_sum)
__device__ __forceinline__ void two_sum2(unsigned long long a, unsigned long long b, unsigned long long &s,
                                         unsigned long long &e)
{
    s = fadd2(a, b);
    const unsigned long long bb = fsub2(s, a);
    e = fadd2(fsub2(a, fsub2(s, bb)), fsub2(b, bb));
}
enum { A_SHI = 0, A_SLO, A_DHI, A_DLO, A_A, A_E, A_ALO };

// 8-byte asynchronous global -> shared copy (completion: cp_async_wait_all by the issuing thread)
// float-float arithmetic on both lanes of packed pairs: each lane performs exactly the IEEE
// operations of the scalar ff_add / ff_sub / ff_mul (lr_mixed.cuh), so results are identical
struct ff2 {
    unsigned long long hi, lo;
};

__device__ __forceinline__ ff2 fast_two_sum2(unsigned long long a, unsigned long long b)
{
    const unsigned long long s = fadd2(a, b);
    return {s, fsub2(b, fsub2(s, a))};
}

__device__ __forceinline__ ff2 ff_add2(ff2 a, ff2 b)
{
    unsigned long long s, e;
    two_sum2(a.hi, b.hi, s, e);
    return fast_two_sum2(s, fadd2(e, fadd2(a.lo, b.lo)));
}

// a - b as a + (-b): the negation is exact, so each operation below rounds as its scalar
// counterpart with the negated operand
__device__ __forceinline__ ff2 ff_sub2(ff2 a, ff2 b)
{
    const unsigned long long s = fsub2(a.hi, b.hi);
    const unsigned long long bb = fsub2(s, a.hi);
    const unsigned long long e = fsub2(fsub2(a.hi, fsub2(s, bb)), fadd2(b.hi, bb));
    return fast_two_sum2(s, fadd2(e, fsub2(a.lo, b.lo)));
}

__device__ __forceinline__ ff2 ff_mul2(ff2 a, ff2 b)
{
    const unsigned long long p = fmul2(a.hi, b.hi);
    unsigned long long e = ffma2(a.hi, b.hi, fneg2(p));
    e = ffma2(a.hi, b.lo, e);
    e = ffma2(a.lo, b.hi, e);
    return fast_two_sum2(p, e);
}

}  // namespace lr
