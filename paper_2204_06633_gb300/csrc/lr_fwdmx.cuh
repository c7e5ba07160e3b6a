// Mixed-precision forward kernels (FP32 taps and accumulation of the interpolated strain,
// float-float link series and TDI sums, FP64 for times, the orbit splines and the delays).
//
// A CTA of 256 threads walks tiles of output samples; per tile it runs these phases, each
// ended by a barrier:
//  setup    FP64: each of the 9 strain read positions (3 reception reads, 6 emission reads,
//           Eq. for y_slr) and each of the 6 link delays re-expanded from the orbit spline as a
//           cubic around the tile centre, held as a 64-bit fixed-point value and slope plus an
//           FP32 remainder polynomial; 12 geometry factors den_l xi_l sampled for a cubic fit.
//  stage    the strain window (TDI-only launches: the link series) in FP64 and its maximum;
//           the reference fraction of every delayed TDI term and its correction weights.
//  convert  scaled by a power of two to float-float, in the 8-phase layout.
//  tables   first, second and third differences of the staged series (two series per thread on
//           the lanes of packed f32x2 pairs).
//  project  work item = one read position x 8 consecutive samples: exact fixed-point positions
//           and index splits, one set of correction weights and its exact derivative per item
//           (the fraction drifts by the Doppler rate ~1e-4 per sample), an FIR over a register
//           window of third differences, a float-float anchor; both polarisations.
//  links    y_l = c+_l (h+(emission) - h+(reception)) + cx_l (hx(emission) - hx(reception)) in
//           float-float, in place, two links with a common receiver per packed pair; the
//           per-sample link delays of the tile in fixed point.
//  tables   of the six link series (three pairs).
//  TDI      work item = one channel x 4 consecutive outputs: both Michelson chains summed into
//           one compensated accumulator; each delayed read uses the tile reference weights and
//           their derivative (a first-order expansion in the fraction, which drifts by ~1e-7 per
//           sample), a register window of third differences and a float-float anchor.
//           Nested chained delays add a per-tile constant per term (nested minus summed delay,
//           from the plan's knot table).
//  like     (KIND_LIKE only) A, E, T of the tile against the data, fetched by cp.async during
//           the TDI phase; FP32 products on the tile-scaled values, a fixed-order block sum.
// Reads whose integer index does not follow the item's pattern (an index step inside an item,
// a knot of the orbit spline inside a projection item) take an exact per-sample path.
#pragma once
#include <cuda_runtime.h>
#include <limits.h>

#include "lr_device.cuh"
#include "lr_mixed.cuh"
#include "lr_tdi_table.cuh"

namespace lr {
// internal linkage: every file that instantiates kernels keeps its own copies of these helpers
namespace {

__constant__ TdiTab c_tdimx = make_tdi_tab();

constexpr int NTERM = 42;  // 3 channels x 2 chains x 7 delayed terms
constexpr float TAU_UNIT = 0x1p-10f;
constexpr int PB = 8;             // samples per projection item
constexpr int TB = MX_TDI_BLOCK;  // outputs per TDI item
constexpr int RLW = MX_AW / 8, RLY = MX_AY / 8;
// shared-memory regions (floats)
constexpr int OFF_W = 0;                    // strain tables: 2 polarisations x 7 arrays
constexpr int OFF_Y = 14 * MX_AW;           // link tables 6 x 6 arrays (staged reads before them)
constexpr int OFF_TW = OFF_Y + 36 * MX_AY;  // TDI correction weights (U, dU/deps) per term
// delay tables of a tile's outputs (in the strain region once the projection is done): the link
// delay at the first output of each TDI item (int64, fixed point) and the increments within
// the item (FP32: differences of at most 3 samples, exact integers in units of 2^-44)
constexpr int LB = MX_YCAP / TB;  // items per row
constexpr int LT = MX_YCAP;       // outputs per row
static_assert(OFF_TW % 4 == 0, "weights must be 16-byte aligned");
static_assert(2 * MX_WCAP * 2 <= 36 * MX_AY, "FP64 strain staging fits the link region");
static_assert(6 * MX_YCAP * 2 <= 14 * MX_AW, "FP64 link staging fits the strain region");
static_assert(6 * LB * 2 + 6 * LT <= 14 * MX_AW, "the delay tables fit the strain region");
// X, Y, Z of a tile for the likelihood epilogue (scaled FP32, after the delay tables) ...
constexpr int XYZ_CAP = MX_TDI_BLOCK * (MIXED_THREADS / 3);  // largest mixed tile
constexpr int OFF_XYZ = OFF_W + 6 * LB * 2 + 6 * LT;
// and the tile's A, E, T data (FP64)
constexpr int OFF_LD = OFF_XYZ + 3 * XYZ_CAP;
static_assert(OFF_LD % 2 == 0 && OFF_LD + 2 * 3 * XYZ_CAP <= OFF_W + 14 * MX_AW,
              "the likelihood staging fits the strain region after the delay tables");

__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Likelihood terms of one output sample in FP32 on values scaled by the tile scale 2^se (the
// template X, Y, Z and the data dA, dE, dT), weights normalised to the largest one
__device__ __forceinline__ void like_terms_f(const LikeArgs &L, float X, float Y, float Z, float dA, float dE,
                                             float dT, float &dh, float &hh)
{
    const float s = X + Z;
    const float a = (Z - X) * 0.70710678f, e = fmaf(-2.0f, Y, s) * 0.40824829f, t = (s + Y) * 0.57735027f;
    const float wa = L.wn[0] * a, we = L.wn[1] * e, wt = L.wn[2] * t;
    dh = fmaf(wa, dA, fmaf(we, dE, fmaf(wt, dT, dh)));
    hh = fmaf(wa, a, fmaf(we, e, fmaf(wt, t, hh)));
}

// Block sum of (a, b) in FP32 in a fixed order (shuffle tree, then the warps in index order);
// thread 0 gets the sums
__device__ __forceinline__ void block_sum2f(float &a, float &b, float *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[2 * w] = a;
        red[2 * w + 1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float sa = 0.0f, sb = 0.0f;
        for (int i = 0; i < MIXED_THREADS / 32; ++i) {
            sa += red[2 * i];
            sb += red[2 * i + 1];
        }
        a = sa;
        b = sb;
    }
}

__device__ __forceinline__ int phw(int j) { return (j & 7) * RLW + (j >> 3); }
__device__ __forceinline__ int phy(int j) { return (j & 7) * RLY + (j >> 3); }
__host__ __device__ constexpr int warr(int pol, int k) { return OFF_W + (7 * pol + k) * MX_AW; }
__device__ __forceinline__ int ybase(int l) { return OFF_Y + 6 * l * MX_AY; }

// x(j) = Xc + (j - jc) Vc + rem(r),  rem(r) = r (v + r (a2 + r a3)),  r = j - jc, in units of 2^-44
struct PosPiece {
    long long Xc, Vc;
    float v, a2, a3, pad;
};

// Everything a tile's compute phases need from its setup: double-buffered, so the setup of a
// CTA's next tile can run while the current one is processed.
struct TileSetup {
    TileInfo ti;
    SkyConst sk;
    int64_t k_lo;  // first sample of the link span
    int ny;        // link span (outputs + TDI halo)
    double u0;     // strain index of output sample 0
    int wlo, whi;  // extent of the read positions over the span (tile-local samples)
    // read positions: [piece][read], tile-local (strain index - k_lo)
    PosPiece pp[2][9];
    int jsw, jc;
    // link delays in samples: [piece][link], output-local index
    PosPiece dp[2][6];
    int jswt, ic;
    // geometry factors c+_l, cx_l at the Chebyshev nodes of tau = (j - jc) 2^-10, and as cubics
    // in tau (constant in float-float)
    double gnode[4][12];
    double tmax, inv_tmax;
    float g0h[12], g0l[12], g1h[12], g1l[12], g2[12], g3[12];
    // maximum of the tile's raw inputs (bit pattern)
    unsigned long long maxbits;
};

struct __align__(16) TermRef {
    long long dnest;
    int tfm;
    float tehi;
};

struct MxShared {
    TileSetup ts[2];
    int64_t tot;     // tiles of the launch
    int64_t s_hint;  // source of the CTA's latest tile
    int unscale_e;   // exponent of the inverse of the current tile's power-of-two scale
    // TDI reference per delayed term (current tile)
    // per delayed term: nested minus summed total delay at the reference output (fixed point,
    // constant over a tile; 0 for summed delays), the reference index offset and fraction
    TermRef tref[NTERM];
    // per delayed term, for the items of even and odd index b: the shared-memory offsets of the
    // third-difference entries x .. x + 7 of the term's fast-path window start x = 4 b + HL +
    // tfm - h, less b / 2 (the link array's base and the 8-phase layout folded in)
    int4 toff[NTERM][2][2];
    float redf[2 * (MIXED_THREADS / 32)];  // likelihood block sums
};

// setup lanes: read-position and link-delay pieces on the first 30 lanes of warp 6, geometry
// nodes on the first 12 of warp 7 (in fused and projection launches these warps have one
// projection item and are free for the next tile's setup while the others finish theirs)
constexpr int SETUP_PIECE0 = 192, SETUP_GEO0 = 224;
// TDI reference lanes of fused launches: a link span holds at most MX_YCAP <= 2 x 256 - 128
// samples, so threads 128 .. 169 have one sample of the link loop and are free for a second
static_assert(MX_YCAP <= MIXED_THREADS + 128, "the TDI reference lanes have a single link sample");
constexpr int TDI_REF0 = 128;

// ---------------------------------------------------------------- helpers
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

// knot-piece switch: first index of [0, n) that lies in the piece after the one at index 0
__device__ inline int piece_switch(double ua, double rstep, int K0, int K1, int n)
{
    if (K1 == K0) return n;
    double jj = ceil(((double)K1 - ua) / rstep);
    return jj < 0 ? 0 : (jj > n ? n : (int)jj);
}

// the cubic c(x), x = xa + j rstep, re-expanded around j = jc in powers of (j - jc):
// value, first, second/2 and third/6 derivative in j
__device__ inline void reexpand(const double *c, double xa, double rstep, int jc, double *d)
{
    const double x = fma((double)jc, rstep, xa);
    d[0] = horner3(c, x);
    d[1] = fma(x, fma(x, 3.0 * c[3], 2.0 * c[2]), c[1]) * rstep;
    d[2] = fma(x, 3.0 * c[3], c[2]) * rstep * rstep;
    d[3] = c[3] * rstep * rstep * rstep;
}

__device__ inline PosPiece make_piece(double P0, double P1, double P2, double P3)
{
    PosPiece p;
    p.Xc = __double2ll_rn(P0 * FX_ONE);
    p.Vc = __double2ll_rn(P1 * FX_ONE);
    p.v = (float)(P1 * FX_ONE - (double)p.Vc);
    p.a2 = (float)(P2 * FX_ONE);
    p.a3 = (float)(P3 * FX_ONE);
    p.pad = 0.0f;
    return p;
}

// remainder of a piece at r = j - jc (rf = r as float)
__device__ __forceinline__ long long piece_rem(const PosPiece &p, float rf)
{
    return (long long)__float2int_rn(rf * fmaf(rf, fmaf(rf, p.a3, p.a2), p.v));
}

__device__ __forceinline__ long long piece_at(const PosPiece &p, int r)
{
    return p.Xc + (long long)r * p.Vc + piece_rem(p, (float)r);
}

// Tile g of the launch: its source, offsets and sky frame.  In a batch the source is found by
// galloping forward from s_hint, the source of the CTA's previous tile (a CTA's tiles come in
// increasing order), then bisecting; the loops are bounded by the 64-bit index width.
__device__ inline void mx_tile(const FwdParams &P, int64_t g, int ochan, int64_t &s_hint, TileInfo &ti,
                               SkyConst &sk)
{
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
        sk = P.src.skyc1;
        if (P.gen_strain) ti.gb = make_gb(P.src.gb1);
    } else {
        const int64_t *to = P.src.tile_off;
        const int64_t S = P.src.S;
        int64_t lo = s_hint;
        if (lo < 0 || lo >= S || __ldg(to + lo) > g) lo = 0;
        int64_t step = 1, hi = lo + 1;
        while (hi < S && __ldg(to + hi) <= g) {  // to[lo] <= g throughout
            lo = hi;
            step <<= 1;
            hi = lo + step;
        }
        if (hi > S) hi = S;
        while (hi - lo > 1) {  // to[lo] <= g < to[hi]
            const int64_t mid = (lo + hi) >> 1;
            if (__ldg(to + mid) <= g) lo = mid; else hi = mid;
        }
        const int64_t s = lo;
        s_hint = s;
        int64_t ho = 0, ho1 = 0;
        if (P.gen_strain) {
            ti.gb = make_gb(P.src.gb[s]);
        } else {
            ho = __ldg(P.src.h_off + s);
            ho1 = __ldg(P.src.h_off + s + 1);
        }
        const int64_t oo = __ldg(P.src.out_off + s), oo1 = __ldg(P.src.out_off + s + 1);
        ti.N = oo1 - oo;
        ti.nh = ho1 - ho;
        if (ti.N < 0 || ti.nh < 0) ti.ok = 0;
        ti.t0h = P.gen_strain ? P.t0 : __ldg(P.src.t0h + s);  // no strain arrays when generated
        ti.sky = P.src.sky[s];
        ti.hp = P.hp + ho;
        ti.hc = P.hc + ho;
        ti.out = P.out ? P.out + ochan * oo : nullptr;
        ti.yin = P.yin ? P.yin + 6 * oo : nullptr;
        ti.dat = like_data(P, oo, oo1);
        ti.n0 = (g - __ldg(to + s)) * P.tile;
        sk = P.src.skyc[s];
    }
    if (P.gen_strain) {  // the waveform on the output grid, at every index
        ti.nh = GEN_STRAIN_LEN;
        ti.t0h = P.t0;
    }
    const int64_t rem = ti.N - ti.n0;
    ti.nb = rem < P.tile ? rem : P.tile;
    if (ti.nb < 0) ti.nb = 0;
}


// block max of the bit patterns b of |v| (for non-negative doubles the order of the patterns is
// the order of the values; a NaN orders above every finite value)
__device__ __forceinline__ unsigned long long abs_bits(double v)
{
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

__device__ inline void block_absmax(unsigned long long *dst, unsigned long long b)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long c = __shfl_xor_sync(0xffffffffu, b, o);
        b = c > b ? c : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(dst, b);
}

// exponent se of the power-of-two scale 2^se putting the tile's largest value in [1/2, 1),
// from the exponent bits of the maximum; 0 for a zero, subnormal or non-finite maximum
__device__ __forceinline__ int tile_scale_exp(unsigned long long maxbits)
{
    const int eb = (int)((maxbits >> 52) & 0x7ffull);  // max = f 2^(eb - 1022), f in [1/2, 1)
    return eb >= 1 && eb <= 2044 ? 1022 - eb : 0;
}

// x 2^se as float-float by integer work on the bit pattern: hi is x's significand rounded to 24
// bits (a carry out of the significand rolls into the exponent field) with the exponent moved by
// se, lo the signed remainder (at most 2^28 units of x's last place, so |lo| <= ulp(hi)/2) as
// FP32.  Values whose scaled hi falls below the FP32 normal range read as zero (below 2^-126 of
// the scaled tile maximum); an infinity or NaN passes through in hi.
__device__ __forceinline__ ff ff_from_double_scaled(double x, int se)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sg = (unsigned)(b >> 32) & 0x80000000u;
    const int ex = (int)((b >> 52) & 0x7ffull);
    const unsigned long long m = b & 0xfffffffffffffull;
    if (ex == 0x7ff) return {__uint_as_float(sg | 0x7f800000u | (m ? 0x400000u : 0u)), 0.0f};
    const int eh = ex - 896 + se;  // FP32 biased exponent of hi (1023 - 127 = 896)
    if (ex == 0 || eh <= 0) return {__uint_as_float(sg), 0.0f};
    if (eh >= 254) return {__uint_as_float(sg | 0x7f800000u), 0.0f};
    const unsigned long long t = m + (1ull << 28);  // round the significand at its 29th bit
    const float hi = __uint_as_float(sg | (((unsigned)eh << 23) + (unsigned)(t >> 29)));
    // remainder r 2^(eh - 127 - 52), r in [-2^28, 2^28); zero once that power leaves the normal
    // range (2^-75 of the scaled maximum at most)
    const int r = (int)((long long)m - (long long)((t >> 29) << 29));
    const int el = eh - 52;
    const float lo = el > 0 ? __int2float_rn(r) * __uint_as_float((unsigned)el << 23) : 0.0f;
    return {hi, sg ? -lo : lo};
}

// f 2^se as a double by integer work (zero and subnormal f read as signed zero: they are below
// 2^-126 of the scaled tile maximum)
__device__ __forceinline__ double f2d_scaled(float f, int se)
{
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    if (e == 0xffu) return (double)f;
    const unsigned long long sgn = (unsigned long long)(b & 0x80000000u) << 32;
    if (e == 0u) return __longlong_as_double((long long)sgn);
    return __longlong_as_double(
        (long long)(sgn | ((unsigned long long)((int)e + 896 + se) << 52) | ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// f 2^k as a double for any k: integer work when the result is a normal double, scalbn otherwise
__device__ __forceinline__ double f2d_pow2(float f, int k)
{
    const int e = (int)((__float_as_uint(f) >> 23) & 0xffu);
    if (e != 0 && e != 0xff && (e + 896 + k < 1 || e + 896 + k > 2046)) return scalbn((double)f, k);
    return f2d_scaled(f, k);
}

// float-float (hi, lo) 2^se as a double: exact conversions of both parts, one FP64 add
__device__ __forceinline__ double ff2d_scaled(float hi, float lo, int se) { return f2d_scaled(hi, se) + f2d_scaled(lo, se); }


// comp_weights_d (lr_mixed.cuh) with its two triple running sums taken on packed (w, dw/deps)
// pairs: W[a] = (U_a, dU_a/deps), each lane the scalar sums, so the values are identical.
template <int T>
__device__ __forceinline__ void comp_weights_d2(float e, unsigned long long *W)
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
    // triple running sums: from the left end left of the centre, from the right end from it on
    unsigned long long s1 = 0ull, s2 = 0ull, s3 = 0ull;
#pragma unroll
    for (int a = 0; a < h; ++a) {
        s1 = fadd2(s1, f2pack(w[a], wd[a]));
        s2 = fadd2(s2, s1);
        s3 = fadd2(s3, s2);
        if (a <= T - 4) W[a] = s3;
    }
    unsigned long long t1 = 0ull, t2 = 0ull, t3 = 0ull, u1[T], u2[T];
#pragma unroll
    for (int a = T - 2; a >= h; --a) {
        t1 = fsub2(t1, f2pack(w[a + 1], wd[a + 1]));
        u1[a] = t1;
    }
#pragma unroll
    for (int a = T - 3; a >= h; --a) {
        t2 = fsub2(t2, u1[a + 1]);
        u2[a] = t2;
    }
#pragma unroll
    for (int a = T - 4; a >= h; --a) {
        t3 = fsub2(t3, u2[a + 1]);
        W[a] = t3;
    }
}

// Difference tables of staged float-float series (arrays at base + k * AS, 8-phase index with
// row length RL): d = s_{j+1} - s_j and a = (d_j - d_{j-1})/2 in float-float (ALO: the low part
// of a kept in its own array, else folded into a), e = d_{j+2} - 2 d_{j+1} + d_j in FP32.
// Two series at once, p and p + npair (series stride SS), on the two lanes of packed pairs, each
// lane the scalar float-float arithmetic; each thread forms Q consecutive entries of a pair from
// one set of differences.  Entries whose stencils leave [0, len) are 0; no read ever uses them.
template <bool ALO, int RL, int Q>
__device__ void build_tables2(float *smf, int base0, int AS, int SS, int npair, int len)
{
    auto at = [](int i) { return (i & 7) * RL + (i >> 3); };
    const int nq = (len + Q - 1) / Q;
    const unsigned long long HALF = f2pack(0.5f, 0.5f);
    for (int it = threadIdx.x; it < npair * nq; it += blockDim.x) {
        const int pr = it / nq, t = it - pr * nq;
        const int b0 = base0 + pr * SS, b1 = base0 + (pr + npair) * SS;
        const int j0 = Q * t;
        ff2 s[Q + 4];  // s_{j0-1} .. s_{j0+Q+2}
#pragma unroll
        for (int u = 0; u < Q + 4; ++u) {
            const int i = j0 - 1 + u;
            const bool in = i >= 0 && i < len;
            const int p = in ? at(i) : 0;
            s[u] = in ? ff2{f2pack(smf[b0 + p], smf[b1 + p]), f2pack(smf[b0 + AS + p], smf[b1 + AS + p])}
                      : ff2{0ull, 0ull};
        }
        ff2 d[Q + 3], dd[Q + 2];
#pragma unroll
        for (int u = 0; u < Q + 3; ++u) d[u] = ff_sub2(s[u + 1], s[u]);
#pragma unroll
        for (int u = 0; u < Q + 2; ++u) dd[u] = ff_sub2(d[u + 1], d[u]);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int j = j0 + k;
            if (j >= len) break;
            unsigned long long DH = 0ull, DL = 0ull, A = 0ull, AL = 0ull, E = 0ull;
            if (j + 1 < len) {
                DH = d[k + 1].hi;
                DL = d[k + 1].lo;
                if (j >= 1) {
                    A = fmul2(HALF, dd[k].hi);
                    AL = fmul2(HALF, dd[k].lo);
                }
                if (j + 3 < len) {
                    const ff2 e3 = ff_sub2(dd[k + 2], dd[k + 1]);
                    E = fadd2(e3.hi, e3.lo);
                }
            }
            const int p = at(j);
            float x0, x1;
            f2unpack(DH, x0, x1);
            smf[b0 + A_DHI * AS + p] = x0;
            smf[b1 + A_DHI * AS + p] = x1;
            f2unpack(DL, x0, x1);
            smf[b0 + A_DLO * AS + p] = x0;
            smf[b1 + A_DLO * AS + p] = x1;
            f2unpack(E, x0, x1);
            smf[b0 + A_E * AS + p] = x0;
            smf[b1 + A_E * AS + p] = x1;
            if (ALO) {
                f2unpack(A, x0, x1);
                smf[b0 + A_A * AS + p] = x0;
                smf[b1 + A_A * AS + p] = x1;
                f2unpack(AL, x0, x1);
                smf[b0 + A_ALO * AS + p] = x0;
                smf[b1 + A_ALO * AS + p] = x1;
            } else {
                f2unpack(fadd2(A, AL), x0, x1);
                smf[b0 + A_A * AS + p] = x0;
                smf[b1 + A_A * AS + p] = x1;
            }
        }
    }
}

// Generated strain window of a tile (Galactic binary on the output grid): out of line, so the
// double-double phase and the sincos stay out of the hot body of kernels that read strain arrays.
// Samples j0, j0 + stride, ...; returns this thread's largest bit pattern of |h|.
__device__ __noinline__ unsigned long long stage_generated(const GbConst &g, double t0, double dt, int64_t i0,
                                                           int wlen, double *pf, int j0, int stride)
{
    unsigned long long mx = 0ull;
    for (int j = j0; j < wlen; j += stride) {
        double a, b;
        gb_strain(g, t0, dt, i0 + j, a, b);
        pf[j] = a;
        pf[MX_WCAP + j] = b;
        mx = max(mx, max(abs_bits(a), abs_bits(b)));
    }
    return mx;
}

// ---------------------------------------------------------------- per-tile setup
// Tile g's bookkeeping (one thread): source, offsets, sky frame, span.
template <int KIND>
__device__ void tile_begin(const FwdParams &P, MxShared &sh, TileSetup &ts, int64_t g)
{
    mx_tile(P, g, KIND == KIND_PROJECT ? 6 : 3, sh.s_hint, ts.ti, ts.sk);
    if (!ts.ti.ok) atomicOr(P.err, ERR_OFFSETS);
    const int hl = KIND == KIND_PROJECT ? 0 : P.HL, hr = KIND == KIND_PROJECT ? 0 : P.HR;
    ts.k_lo = ts.ti.n0 - hl;
    ts.ny = (int)ts.ti.nb + hl + hr;
    ts.u0 = (P.t0 - ts.ti.t0h) * P.inv_dt;
    ts.wlo = INT_MAX;
    ts.whi = INT_MIN;
    ts.maxbits = 0ull;
    ts.tmax = ((double)(ts.ny / 2) + 1.0) * (double)TAU_UNIT;
    ts.inv_tmax = 1.0 / ts.tmax;
    if (ts.ny > MX_YCAP) {
        atomicOr(P.err, ERR_WINDOW);
        ts.ti.ok = 0;
    }
}

// Setup lane task t in [0, 30): t < 18 the read-position piece [t / 9][read t % 9] with the
// span's position extent, t >= 18 the link-delay piece [(t - 18) / 6][link (t - 18) % 6].  Both
// are a cubic c(x) = sum of up to four weighted orbit series on one knot interval, re-expanded
// around the centre sample: positions j + u0 - c, delays c (samples).  One code path, so the
// 30 tasks cost one warp's FP64 instruction stream.
template <int KIND>
__device__ void setup_piece(const FwdParams &P, TileSetup &ts, int t)
{
    const bool pos = t < 18;
    if (pos ? KIND == KIND_TDI : KIND == KIND_PROJECT) return;
    const OrbitDev &o = pos ? P.po : P.to;
    const int n = pos ? ts.ny : (int)ts.ti.nb;
    const int64_t s0 = pos ? ts.k_lo : ts.ti.n0;
    const double rstep = P.dt * o.inv_dk;
    const double ua = (P.t0 + (double)s0 * P.dt - o.t_first) * o.inv_dk;
    const double ub = ua + (double)(n - 1) * rstep;
    const int K0 = clampK(o, ua), K1 = clampK(o, ub);
    const int sw = piece_switch(ua, rstep, K0, K1, n);
    const int u = pos ? t : t - 18;
    const int iv = pos ? u / 9 : u / 6;
    const int K = iv == 0 ? K0 : K1;
    // emission reads (rd >= 3) of link l = rd - 3 shift by the emitter's k.x/c and L_l;
    // reception reads by the receiver's k.x/c
    int ser[4];
    double w[4];
    int nt;
    if (pos) {
        const int rd = u % 9;
        const int sc = rd < 3 ? rd : (rd == 3 ? 1 : rd == 4 ? 2 : rd == 5 ? 0 : rd == 6 ? 2 : rd == 7 ? 1 : 0);
        const double kc = P.inv_dt * (1.0 / C_LIGHT);
        for (int d = 0; d < 3; ++d) {
            ser[d] = 3 * sc + d;
            w[d] = ts.sk.k[d] * kc;
        }
        ser[3] = 9 + (rd >= 3 ? rd - 3 : 0);
        w[3] = P.inv_dt;
        nt = rd >= 3 ? 4 : 3;
    } else {
        ser[0] = 9 + u % 6;
        w[0] = P.inv_dt;
        ser[1] = ser[2] = ser[3] = 0;
        w[1] = w[2] = w[3] = 0.0;
        nt = 1;
    }
    double c[4] = {0.0, 0.0, 0.0, 0.0};
    for (int v = 0; v < nt; ++v) {
        const double *q = orbit_coef_ptr(o, K, ser[v]);
        for (int i = 0; i < 4; ++i) c[i] = fma(w[v], q[i], c[i]);
    }
    const int cen = n / 2;
    double d[4];
    reexpand(c, ua - (double)K, rstep, cen, d);
    const double sg = pos ? -1.0 : 1.0;
    const PosPiece pc = make_piece(fma(sg, d[0], pos ? (double)cen + ts.u0 : 0.0), fma(sg, d[1], pos ? 1.0 : 0.0),
                                   sg * d[2], sg * d[3]);
    if (pos) {
        ts.pp[iv][u % 9] = pc;
        // extent of the positions (increasing in j) at the span ends, on the piece holding them
        // (a position outside +-2^18 samples, never a valid one, marks the window as too wide)
        const long long lim = 1ll << (FX_BITS + 18);
        if ((0 < sw) == (iv == 0)) {
            const long long X = piece_at(pc, -cen);
            atomicMin(&ts.wlo, X > -lim && X < lim ? (int)(X >> FX_BITS) : INT_MIN / 2);
        }
        if ((n - 1 < sw) == (iv == 0)) {
            const long long X = piece_at(pc, n - 1 - cen);
            atomicMax(&ts.whi, X > -lim && X < lim ? (int)(X >> FX_BITS) : INT_MAX / 2);
        }
        if (u == 0) {
            ts.jsw = sw;
            ts.jc = cen;
        }
    } else {
        ts.dp[iv][u % 6] = pc;
        if (u == 0) {
            ts.jswt = sw;
            ts.ic = cen;
        }
    }
}

// geometry factors of arm a at Chebyshev node i (Eq. projected-strain-ssb patterns, psi
// rotation, 1/(2(1 -+ k.n)) for the two directions); task f = 3 i + a in [0, 12)
__device__ void setup_geometry(const FwdParams &P, TileSetup &ts, int f)
{
    const OrbitDev &o = P.po;
    const int i = f / 3, a = f % 3;
    const double tau = ts.tmax * P.cheb_node[i];
    const double t = P.t0 + ((double)(ts.k_lo + ts.ny / 2) + tau / (double)TAU_UNIT) * P.dt;
    double x;
    const Coef4 *row = spline_row(o, t, &x);
    const int r = a, s = (a + 1) % 3;
    double d[3];
    for (int c = 0; c < 3; ++c) d[c] = cubic(ldg4(row + 3 * r + c), x) - cubic(ldg4(row + 3 * s + c), x);
    const SkyConst &S = ts.sk;
    const double inv = rsqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const double n0 = d[0] * inv, n1 = d[1] * inv, n2 = d[2] * inv;
    const double un = S.u[0] * n0 + S.u[1] * n1 + S.u[2] * n2;
    const double vn = S.v[0] * n0 + S.v[1] * n1 + S.v[2] * n2;
    const double kn = S.k[0] * n0 + S.k[1] * n1 + S.k[2] * n2;
    const double xip = un * un - vn * vn, xic = 2.0 * un * vn;
    const double xp = S.c2p * xip + S.s2p * xic, xc = -S.s2p * xip + S.c2p * xic;
    // 1/(2(1 - kn)) and 1/(2(1 + kn)) from one division
    const double den = 0.5 / ((1.0 - kn) * (1.0 + kn));
    const double df = (1.0 + kn) * den, dr = (1.0 - kn) * den;
    ts.gnode[i][a] = xp * df;
    ts.gnode[i][6 + a] = xc * df;
    ts.gnode[i][5 - a] = xp * dr;
    ts.gnode[i][11 - a] = xc * dr;
}

// cubic through the 4 geometry nodes: monomial coefficients in tau from the Chebyshev
// inverse Vandermonde (factor f)
__device__ void fit_geometry(const FwdParams &P, TileSetup &ts, int f)
{
    double b[4];
    double sc = 1.0;
    for (int k = 0; k < 4; ++k) {
        double acc = 0.0;
        for (int i = 0; i < 4; ++i) acc = fma(P.cheb[k][i], ts.gnode[i][f], acc);
        b[k] = acc * sc;
        sc *= ts.inv_tmax;
    }
    const ff c0 = ff_from_double(b[0]), c1 = ff_from_double(b[1]);
    ts.g0h[f] = c0.hi;
    ts.g0l[f] = c0.lo;
    ts.g1h[f] = c1.hi;
    ts.g1l[f] = c1.lo;
    ts.g2[f] = (float)b[2];
    ts.g3[f] = (float)b[3];
}

// the setup lanes of a tile (see SETUP_PIECE0); warp 7 fits the geometry cubics once its 12
// lanes have the nodes
template <int KIND>
__device__ __forceinline__ void setup_lanes(const FwdParams &P, TileSetup &ts)
{
    const int tid = threadIdx.x;
    if (tid >= SETUP_PIECE0 && tid < SETUP_PIECE0 + 30) {
        setup_piece<KIND>(P, ts, tid - SETUP_PIECE0);
    } else if (KIND != KIND_TDI && tid >= SETUP_GEO0 && tid < SETUP_GEO0 + 32) {
        const int f = tid - SETUP_GEO0;
        if (f < 12) setup_geometry(P, ts, f);
        __syncwarp();
        if (f < 12) fit_geometry(P, ts, f);
    }
}

// Reference of each delayed TDI term at the tile centre ic (its chained delay is the sum of the
// pieces' centre values, exactly what the delay table holds at ic) and the correction weights
// there with their derivative, interleaved as (U_a, dU_a/deps) pairs; threads first ..
// first + 41, one term each.
template <int T>
__device__ void tdi_refs(const FwdParams &P, const TileSetup &ts, MxShared &sh, float *tw, int first)
{
    const int id = threadIdx.x - first;
    if (id < 0 || id >= NTERM) return;
    const int ch = id / 14, c = (id / 7) % 2, q = id % 7 + 1;
    if (q > P.q_terms) return;
    const int iv = ts.ic < ts.jswt ? 0 : 1;
    long long D = 0;
    for (int k = 1; k <= q; ++k) D += ts.dp[iv][c_tdimx.pair[ch][c][k]].Xc;
    // nested chained delays: the nested minus summed total delay of the term at the reference
    // output, interpolated in the plan's knot table (it changes by < 1e-10 samples over a tile,
    // so one value serves the tile; the reference split keeps the summed delay, ~1e-7 samples
    // away: at worst an item leaves the fast path)
    long long dn = 0;
    if (P.nest_tab) {
        const double u = (P.t0 + (double)(ts.ti.n0 + ts.ic) * P.dt - P.nest_t0) * P.nest_inv_dk;
        const int k = u <= 0.0 ? 0 : (u >= (double)(P.nest_n - 2) ? P.nest_n - 2 : (int)u);
        const double f = fmin(fmax(u - (double)k, 0.0), 1.0);
        const double a = __ldg(P.nest_tab + k * NTERM + id), b = __ldg(P.nest_tab + (k + 1) * NTERM + id);
        dn = llrint(fma(f, b - a, a) * (double)(1ll << FX_BITS));
    }
    sh.tref[id].dnest = dn;
    const int nlr = ts.ic + P.HL;
    const Split s = split_fx(((long long)nlr << FX_BITS) - D);
    sh.tref[id].tfm = s.m - nlr;
    sh.tref[id].tehi = s.ehi;
    {
        const int yb = ybase(c_tdimx.link[ch][c][q]) + A_E * MX_AY;
        const int K = P.HL + (s.m - nlr) - (T - 2) / 2;
        int o[16];
#pragma unroll
        for (int par = 0; par < 2; ++par)
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int v = 4 * par + K + r;  // floor division and modulo by shift and mask
                o[8 * par + r] = yb + (v & 7) * RLY + (v >> 3);
            }
#pragma unroll
        for (int par = 0; par < 2; ++par) {
            sh.toff[id][par][0] = make_int4(o[8 * par], o[8 * par + 1], o[8 * par + 2], o[8 * par + 3]);
            sh.toff[id][par][1] = make_int4(o[8 * par + 4], o[8 * par + 5], o[8 * par + 6], o[8 * par + 7]);
        }
    }
    constexpr int NUP = mx_nup(T);
    float2 *w = reinterpret_cast<float2 *>(tw) + id * NUP;
    if constexpr (T >= 4) {
        constexpr int NU = T - 3;
        unsigned long long W[NU];
        comp_weights_d2<T>(s.ehi, W);
#pragma unroll
        for (int a = 0; a < NUP; ++a) {
            float u = 0.0f, u1 = 0.0f;
            if (a < NU) f2unpack(W[a], u, u1);
            w[a] = make_float2(u, u1);
        }
    } else {
#pragma unroll
        for (int a = 0; a < NUP; ++a) w[a] = make_float2(0.0f, 0.0f);
    }
}

// ---------------------------------------------------------------- projection reads
// float-float s + eps d + eps (eps - 1) a - C of a strain series at 8-phase position ai (the
// curvature product formed from the exact eps_hi (eps_hi - 1) against the float-float a: it
// feeds two levels of cancellation).  The result is an unnormalised float-float pair.  Degree 1
// (T = 2) is the linear anchor s + eps d alone.
template <int T>
__device__ __forceinline__ ff strain_anchor(const float *smf, int pol, int ai, float eh, float el, float C)
{
    if constexpr (T < 4) {
        const float shi = smf[warr(pol, A_SHI) + ai], slo = smf[warr(pol, A_SLO) + ai];
        const float dhi = smf[warr(pol, A_DHI) + ai], dlo = smf[warr(pol, A_DLO) + ai];
        const float p = eh * dhi;
        const float pe = fmaf(eh, dhi, -p);
        const ff t1 = two_sum(shi, p);
        return {t1.hi, (slo + t1.lo) + (pe + fmaf(eh, dlo, el * dhi))};
    }
    const float shi = smf[warr(pol, A_SHI) + ai], slo = smf[warr(pol, A_SLO) + ai];
    const float dhi = smf[warr(pol, A_DHI) + ai], dlo = smf[warr(pol, A_DLO) + ai];
    const float ahi = smf[warr(pol, A_A) + ai], alo = smf[warr(pol, A_ALO) + ai];
    const float p = eh * dhi;
    const float pe = fmaf(eh, dhi, -p);
    const float em1 = eh - 1.0f;
    const float q = eh * em1;
    const float qe = fmaf(el, 2.0f * eh - 1.0f, fmaf(eh, em1, -q));
    const float cq = q * ahi;
    const float cqe = fmaf(q, ahi, -cq);
    const ff t1 = two_sum(shi, p);
    const ff t2 = two_sum(t1.hi, cq);
    const float lo = (slo + (t1.lo + t2.lo)) + (pe + fmaf(eh, dlo, el * dhi)) + (cqe + fmaf(q, alo, qe * ahi)) - C;
    return {t2.hi, lo};
}

// strain_anchor on a pair of samples at once (packed lanes; per lane the same arithmetic as the
// scalar form with the signs of intermediate error terms carried negated, which rounds
// identically): EH, EL, NEH = -EH of the two samples, C their correction sums; returns the
// unnormalised float-float pairs (HI, LO)
template <int T>
__device__ __forceinline__ void strain_anchor2(const float *smf, int pol, int a0, int a1, unsigned long long EH,
                                               unsigned long long NEH, unsigned long long EL, unsigned long long C,
                                               unsigned long long &HI, unsigned long long &LO)
{
    auto ld = [&](int arr) { return f2pack(smf[warr(pol, arr) + a0], smf[warr(pol, arr) + a1]); };
    const unsigned long long SHI = ld(A_SHI), SLO = ld(A_SLO), DHI = ld(A_DHI), DLO = ld(A_DLO);
    const unsigned long long Pp = fmul2(EH, DHI);
    const unsigned long long NPE = ffma2(NEH, DHI, Pp);  // -(eh dhi - p)
    unsigned long long S1, E1;
    two_sum2(SHI, Pp, S1, E1);
    const unsigned long long LIN = fsub2(ffma2(EH, DLO, fmul2(EL, DHI)), NPE);
    if constexpr (T < 4) {
        HI = S1;
        LO = fadd2(fadd2(SLO, E1), LIN);
    } else {
        const unsigned long long AHI = ld(A_A), ALO = ld(A_ALO);
        const unsigned long long ONE = f2pack(1.0f, 1.0f);
        const unsigned long long EM1 = fsub2(EH, ONE);
        const unsigned long long Q = fmul2(EH, EM1);
        const unsigned long long NQ = fmul2(NEH, EM1);                                 // -q exactly
        const unsigned long long NQE0 = ffma2(NEH, EM1, Q);                            // -(eh em1 - q)
        const unsigned long long G = ffma2(f2pack(2.0f, 2.0f), EH, fneg2(ONE));        // 2 eh - 1
        const unsigned long long QE = ffma2(EL, G, fneg2(NQE0));
        const unsigned long long CQ = fmul2(Q, AHI);
        const unsigned long long NCQE = ffma2(NQ, AHI, CQ);                            // -(q ahi - cq)
        unsigned long long S2, E2;
        two_sum2(S1, CQ, S2, E2);
        HI = S2;
        const unsigned long long CUR = fsub2(ffma2(Q, ALO, fmul2(QE, AHI)), NCQE);
        LO = fsub2(fadd2(fadd2(fadd2(SLO, fadd2(E1, E2)), LIN), CUR), C);
    }
}

__device__ __forceinline__ void store_read(float *smf, int rd, int pol, int j, ff v)
{
    const int row = rd * 4 + pol * 2;
    smf[OFF_Y + row * MX_AY + phy(j)] = v.hi;
    smf[OFF_Y + (row + 1) * MX_AY + phy(j)] = v.lo;
}

// One projection item sample by sample with exact weights: items whose integer index steps
// inside the item, or that straddle a knot of the orbit spline.  Out-of-window stencils read 0
// and record ERR_WINDOW.
template <int T>
__device__ __noinline__ void proj_item_exact(float *smf, const TileSetup &sh, int rd, int j0, int kmax, int wlen,
                                             long long woff_fx, int *err)
{
    constexpr int h = (T - 2) / 2;
    for (int k = 0; k < kmax; ++k) {
        const int j = j0 + k;
        const PosPiece p = sh.pp[j < sh.jsw ? 0 : 1][rd];
        const Split s = split_fx(piece_at(p, j - sh.jc) - woff_fx);
        if (s.m - h < 0 || s.m + h + 1 >= wlen) {
            atomicOr(err, ERR_WINDOW);
            store_read(smf, rd, 0, j, {0.0f, 0.0f});
            store_read(smf, rd, 1, j, {0.0f, 0.0f});
            continue;
        }
        float U[T >= 4 ? T - 3 : 1];
        if constexpr (T >= 4) comp_weights<T>(s.ehi, U);
        for (int pol = 0; pol < 2; ++pol) {
            float C = 0.0f;
            if constexpr (T >= 4) {
#pragma unroll
                for (int a = 0; a < T - 3; ++a) C = fmaf(U[a], smf[warr(pol, A_E) + phw(s.m - h + a)], C);
            }
            store_read(smf, rd, pol, j, strain_anchor<T>(smf, pol, phw(s.m), s.ehi, s.elo, C));
        }
    }
}

// Projection item: read rd at the samples j0 .. j0+7 of the span.
template <int T>
__device__ __forceinline__ void proj_item(float *smf, const TileSetup &sh, int rd, int b, int ny, int wlen,
                                          long long woff_fx, int *err)
{
    constexpr int h = (T - 2) / 2;
    constexpr int NU = T >= 4 ? T - 3 : 1;
    constexpr int NE = NU + PB - 1;
    const int j0 = PB * b;
    const int kmax = min(PB, ny - j0);
    const int piece = j0 < sh.jsw ? 0 : 1;
    if (piece == 0 && j0 + kmax - 1 >= sh.jsw) {
        proj_item_exact<T>(smf, sh, rd, j0, kmax, wlen, woff_fx, err);
        return;
    }
    float eh[PB], el[PB];
    int m0;
    bool steady = true;
    {
        const PosPiece p = sh.pp[piece][rd];
        const int r0 = j0 - sh.jc;
        const float rf0 = (float)r0;
        long long X = p.Xc + (long long)r0 * p.Vc - woff_fx;
        int mk0 = 0;
#pragma unroll
        for (int k = 0; k < PB; ++k) {
            const Split s = split_fx(X + piece_rem(p, rf0 + (float)k));
            if (k == 0)
                mk0 = s.m;
            else if (k < kmax)
                steady = steady && (s.m == mk0 + k);
            eh[k] = s.ehi;
            el[k] = s.elo;
            X += p.Vc;
        }
        m0 = mk0;
    }
    if (!steady) {
        proj_item_exact<T>(smf, sh, rd, j0, kmax, wlen, woff_fx, err);
        return;
    }
    if (m0 - h < 0 || m0 + kmax + h >= wlen) {
        atomicOr(err, ERR_WINDOW);
        for (int k = 0; k < kmax; ++k) {
            store_read(smf, rd, 0, j0 + k, {0.0f, 0.0f});
            store_read(smf, rd, 1, j0 + k, {0.0f, 0.0f});
        }
        return;
    }
    // 8-phase offsets of the window start x = m0 - h: element a sits at o[a % 8] + a / 8
    const int x = m0 - h;
    int o[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) o[r] = phw(x + r);
    const float eref = kmax == PB ? eh[PB / 2] : eh[0];
    // correction weights and their derivative as packed (U_a, dU_a/deps) pairs
    unsigned long long W[NU];
    if constexpr (T >= 4) comp_weights_d2<T>(eref, W);
#pragma unroll 1
    for (int pol = 0; pol < 2; ++pol) {
        float C[PB];
        if constexpr (T >= 4) {
            // FIR with packed pairs over a sliding window of (e, e): at tap a the samples
            // k = 0..7 read e[k + a]; only the 8 entries e[a .. a+7] are live
            unsigned long long acc[PB], win[PB];
#pragma unroll
            for (int k = 0; k < PB; ++k) {
                acc[k] = 0ull;
                const float v = smf[warr(pol, A_E) + o[k & 7] + (k >> 3)];
                win[k] = f2pack(v, v);
            }
#pragma unroll
            for (int a = 0; a < NU; ++a) {
#pragma unroll
                for (int k = 0; k < PB; ++k) acc[k] = ffma2(W[a], win[(a + k) % PB], acc[k]);
                if (a + PB < NE) {
                    const int e = a + PB;  // replaces e[a], no longer read
                    const float v = smf[warr(pol, A_E) + o[e & 7] + (e >> 3)];
                    win[a % PB] = f2pack(v, v);
                }
            }
#pragma unroll
            for (int k = 0; k < PB; ++k) {
                float c0, c1;
                f2unpack(acc[k], c0, c1);
                C[k] = fmaf((eh[k] - eref) + el[k], c1, c0);
            }
        } else {
#pragma unroll
            for (int k = 0; k < PB; ++k) C[k] = 0.0f;
        }
#pragma unroll
        for (int pr = 0; pr < PB / 2; ++pr) {
            const int k0 = 2 * pr, k1 = 2 * pr + 1;
            unsigned long long HI, LO;
            strain_anchor2<T>(smf, pol, o[(h + k0) & 7] + ((h + k0) >> 3), o[(h + k1) & 7] + ((h + k1) >> 3),
                              f2pack(eh[k0], eh[k1]), f2pack(-eh[k0], -eh[k1]), f2pack(el[k0], el[k1]),
                              f2pack(C[k0], C[k1]), HI, LO);
            float h0, h1, l0, l1;
            f2unpack(HI, h0, h1);
            f2unpack(LO, l0, l1);
            if (k0 < kmax) store_read(smf, rd, pol, j0 + k0, {h0, l0});
            if (k1 < kmax) store_read(smf, rd, pol, j0 + k1, {h1, l1});
        }
    }
}

// ---------------------------------------------------------------- TDI reads
// sgn * (s + eps d) added to the float-float accumulator (hi, lo) exactly up to the low parts;
// sgn * (eps (eps - 1) a - C) added to the FP32 accumulator sm (T >= 4), with eps = eh + el and
// eps (eps - 1) = q0 + el g (q0 = eh (eh - 1), g = 2 eh - 1).
template <int SG, int T>
__device__ __forceinline__ void acc_term(float &hi, float &lo, float &sm, float shi, float slo, float dhi, float dlo,
                                         float a, float eh, float el, float q0, float g, float C)
{
    const float p = eh * dhi;
    const float pe = fmaf(eh, dhi, -p);
    const ff t1 = two_sum(hi, SG > 0 ? shi : -shi);
    const ff t2 = two_sum(t1.hi, SG > 0 ? p : -p);
    hi = t2.hi;
    const float l = slo + (pe + fmaf(eh, dlo, el * dhi));
    lo += (SG > 0 ? l : -l) + (t1.lo + t2.lo);
    if constexpr (T >= 4) {  // degree 1: the linear anchor alone
        const float c = fmaf(fmaf(el, g, q0), a, -C);
        sm += SG > 0 ? c : -c;
    }
}

// acc_term<1, T> on a pair of outputs at once (packed lanes, each lane the same IEEE operations
// as the scalar form): EH, NEH (= -eh), G, Q0 broadcast; EL, NC (= -C) and the loaded values per
// output
template <int T>
__device__ __forceinline__ void acc_term2(unsigned long long &HI, unsigned long long &LO, unsigned long long &SM,
                                          unsigned long long SHI, unsigned long long SLO, unsigned long long DHI,
                                          unsigned long long DLO, unsigned long long A, unsigned long long EH,
                                          unsigned long long NEH, unsigned long long EL, unsigned long long G,
                                          unsigned long long Q0, unsigned long long NC)
{
    const unsigned long long Pp = fmul2(EH, DHI);
    const unsigned long long NPE = ffma2(NEH, DHI, Pp);  // -(eh dhi - p) exactly rounded: -pe
    unsigned long long S1, E1, S2, E2;
    two_sum2(HI, SHI, S1, E1);
    two_sum2(S1, Pp, S2, E2);
    HI = S2;
    const unsigned long long X = ffma2(EH, DLO, fmul2(EL, DHI));
    const unsigned long long L = fadd2(SLO, fsub2(X, NPE));
    LO = fadd2(LO, fadd2(L, fadd2(E1, E2)));
    if constexpr (T >= 4) SM = fadd2(SM, ffma2(ffma2(EL, G, Q0), A, NC));
}

__device__ __forceinline__ float lane(unsigned long long v, int k)
{
    float a, b;
    f2unpack(v, a, b);
    return k ? b : a;
}

__device__ __forceinline__ void set_lane(unsigned long long &v, int k, float x)
{
    float a, b;
    f2unpack(v, a, b);
    v = k ? f2pack(a, x) : f2pack(x, b);
}

// one delayed read of link lk with exact weights (the rare reads off the tile reference);
// an out-of-window stencil reads 0 and records ERR_WINDOW
template <int T>
__device__ __noinline__ void tdi_read_exact(const float *smf, int lk, int m, float eh, float el, int ny, int *err,
                                            float *out)
{
    constexpr int h = (T - 2) / 2;
    if (m - h < 0 || m + h + 1 >= ny) {
        atomicOr(err, ERR_WINDOW);
        for (int i = 0; i < 6; ++i) out[i] = 0.0f;
        return;
    }
    const int yb = ybase(lk);
    float C = 0.0f;
    if constexpr (T >= 4) {
        float U[T - 3];
        comp_weights<T>(eh, U);
#pragma unroll
        for (int a = 0; a < T - 3; ++a) C = fmaf(U[a], smf[yb + A_E * MX_AY + phy(m - h + a)], C);
    }
    const int ai = phy(m);
    out[0] = smf[yb + A_SHI * MX_AY + ai];
    out[1] = smf[yb + A_SLO * MX_AY + ai];
    out[2] = smf[yb + A_DHI * MX_AY + ai];
    out[3] = smf[yb + A_DLO * MX_AY + ai];
    out[4] = smf[yb + A_A * MX_AY + ai];
    out[5] = C;
}

// Chain c of channel ch, added to the accumulators, for the outputs of item b (i0 = 4 b;
// nl = output index in the span).  The chained delay of the item's first output is carried in 64-bit fixed point
// and split once per term; the other outputs differ from it by the exact FP32 increments
// dk, so output k reads at index m0 + k with fraction eh + (el - dk 2^-44) while that stays
// in [0, 1).
template <int T>
__device__ __forceinline__ void tdi_chain(const FwdParams &P, const MxShared &sh, int ny, const float *smf,
                                          const long long *Lblk, const float *dLf, int ch, int c, int b, int kmax,
                                          unsigned long long *HI, unsigned long long *LO, unsigned long long *SM)
{
    constexpr int h = (T - 2) / 2;
    constexpr int NU = T >= 4 ? T - 3 : 1;
    constexpr int NE = NU + TB - 1;
    constexpr int NUP = mx_nup(T);
    const int i0 = TB * b;
    const int nl0 = i0 + P.HL;
    {
        const int yb = ybase(c_tdimx.link[ch][c][0]);
#pragma unroll
        for (int pr = 0; pr < TB / 2; ++pr) {
            const int a0 = phy(nl0 + 2 * pr), a1 = phy(nl0 + 2 * pr + 1);
            const unsigned long long SHI = f2pack(smf[yb + A_SHI * MX_AY + a0], smf[yb + A_SHI * MX_AY + a1]);
            const unsigned long long SLO = f2pack(smf[yb + A_SLO * MX_AY + a0], smf[yb + A_SLO * MX_AY + a1]);
            unsigned long long S, E;
            two_sum2(HI[pr], SHI, S, E);
            HI[pr] = S;
            LO[pr] = fadd2(LO[pr], fadd2(SLO, E));
        }
    }
    long long D0 = 0;
    float dk[TB];
#pragma unroll
    for (int k = 0; k < TB; ++k) dk[k] = 0.0f;
#pragma unroll 1
    for (int q = 1; q <= P.q_terms; ++q) {
        const int pl = c_tdimx.pair[ch][c][q];
        const int lk = c_tdimx.link[ch][c][q];
        const int id = (ch * 2 + c) * 7 + q - 1;
        D0 += Lblk[pl * LB + b];
        const float4 dv = reinterpret_cast<const float4 *>(dLf + pl * LT)[b];
        dk[1] += dv.y;
        dk[2] += dv.z;
        dk[3] += dv.w;
        const TermRef tr = sh.tref[id];
        const long long Dq = D0 + tr.dnest;  // the term's delay at output i0
        const Split s0 = split_fx(((long long)nl0 << FX_BITS) - Dq);
        const int m0 = s0.m;
        const float eh = s0.ehi;
        float el[TB];
        el[0] = s0.elo;
#pragma unroll
        for (int k = 1; k < TB; ++k) el[k] = fmaf(-dk[k], 0x1p-44f, s0.elo);
        bool fast = (m0 - nl0 == tr.tfm) && (m0 - h >= 0) && (m0 + kmax + h < ny);
#pragma unroll
        for (int k = 1; k < TB; ++k) fast = fast && (k >= kmax || (eh + el[k] >= 0.0f && eh + el[k] < 1.0f));
        const float q0 = eh * (eh - 1.0f), g = 2.0f * eh - 1.0f;
        if (fast) {
            // offsets of the third differences e[x + r] (x = m0 - h), from the tile's table
            const int hb = b >> 1;
            const int4 ta = sh.toff[id][b & 1][0], tb = sh.toff[id][b & 1][1];
            const int o[8] = {hb + ta.x, hb + ta.y, hb + ta.z, hb + ta.w, hb + tb.x, hb + tb.y, hb + tb.z, hb + tb.w};
            float C[TB];
#pragma unroll
            for (int k = 0; k < TB; ++k) C[k] = 0.0f;
            if constexpr (T >= 4) {
                const float dref = eh - tr.tehi;
                // (e, e) pairs of the window in a ring of RW: taps a, a+1 read e[a .. a+TB]
                constexpr int RW = TB + 2;
                unsigned long long win[RW];
#pragma unroll
                for (int a = 0; a < RW; ++a) {
                    const float v = a < NE ? smf[o[a & 7] + (a >> 3)] : 0.0f;
                    win[a] = f2pack(v, v);
                }
                unsigned long long acc[TB];  // (sum U e, sum dU e)
#pragma unroll
                for (int k = 0; k < TB; ++k) acc[k] = 0ull;
                const ulonglong2 *w = reinterpret_cast<const ulonglong2 *>(smf + OFF_TW) + id * (NUP / 2);
#pragma unroll
                for (int a2 = 0; a2 < NUP / 2; ++a2) {
                    const int a = 2 * a2;
                    const ulonglong2 u = w[a2];  // (U, dU) at taps a and a + 1
#pragma unroll
                    for (int k = 0; k < TB; ++k) {
                        acc[k] = ffma2(u.x, win[(a + k) % RW], acc[k]);
                        if (a + 1 < NU) acc[k] = ffma2(u.y, win[(a + 1 + k) % RW], acc[k]);
                    }
#pragma unroll
                    for (int e = a + RW; e < a + RW + 2; ++e)  // e[a], e[a+1] are no longer read
                        if (e < NE) {
                            const float v = smf[o[e & 7] + (e >> 3)];
                            win[e % RW] = f2pack(v, v);
                        }
                }
#pragma unroll
                for (int k = 0; k < TB; ++k) {
                    float c0, c1;
                    f2unpack(acc[k], c0, c1);
                    C[k] = fmaf(dref + el[k], c1, c0);
                }
            }
            const unsigned long long EH = f2pack(eh, eh), NEH = f2pack(-eh, -eh);
            const unsigned long long G2 = f2pack(g, g), Q02 = f2pack(q0, q0);
#pragma unroll
            for (int pr = 0; pr < TB / 2; ++pr) {
                const int k0 = 2 * pr, k1 = 2 * pr + 1;
                const int a0 = o[(h + k0) & 7] + ((h + k0) >> 3), a1 = o[(h + k1) & 7] + ((h + k1) >> 3);
                auto ld = [&](int arr) {
                    return f2pack(smf[(arr - A_E) * MX_AY + a0], smf[(arr - A_E) * MX_AY + a1]);
                };
                acc_term2<T>(HI[pr], LO[pr], SM[pr], ld(A_SHI), ld(A_SLO), ld(A_DHI), ld(A_DLO), ld(A_A), EH, NEH,
                             f2pack(el[k0], el[k1]), G2, Q02, f2pack(-C[k0], -C[k1]));
            }
        } else {
#pragma unroll
            for (int k = 0; k < TB; ++k) {
                if (k < kmax) {
                    const Split sk = split_fx(((long long)(nl0 + k) << FX_BITS) - (Dq + (long long)dk[k]));
                    float r[6];
                    tdi_read_exact<T>(smf, lk, sk.m, sk.ehi, sk.elo, ny, P.err, r);
                    float hk = lane(HI[k >> 1], k & 1), lk_ = lane(LO[k >> 1], k & 1), sk_ = lane(SM[k >> 1], k & 1);
                    acc_term<1, T>(hk, lk_, sk_, r[0], r[1], r[2], r[3], r[4], sk.ehi, sk.elo,
                                   sk.ehi * (sk.ehi - 1.0f), 2.0f * sk.ehi - 1.0f, r[5]);
                    set_lane(HI[k >> 1], k & 1, hk);
                    set_lane(LO[k >> 1], k & 1, lk_);
                    set_lane(SM[k >> 1], k & 1, sk_);
                }
            }
        }
    }
}

// ---------------------------------------------------------------- kernel
template <int T, int KIND>
__global__ void __launch_bounds__(MIXED_THREADS, (T <= 32 ? 2 : 1)) k_mixed(FwdParams P)
{
    extern __shared__ __align__(16) float smf[];
    __shared__ MxShared sh;
    constexpr int h = (T - 2) / 2;
    // fused and projection launches set up the CTA's next tile on the warps a projection phase
    // leaves idle; TDI-only launches set up each tile in place
    constexpr bool PREFETCH = KIND != KIND_TDI;
    constexpr bool LIKE = KIND == KIND_LIKE;                 // fused + likelihood epilogue
    constexpr bool FUSED = KIND == KIND_FUSED || LIKE;
    const int tid = threadIdx.x;
    if (tid == 0) {
        sh.tot = P.total_tiles >= 0 ? P.total_tiles : P.src.tile_off[P.src.S];
        sh.s_hint = 0;
    }
    __syncthreads();
    int cur = 0;
    if (PREFETCH && blockIdx.x < sh.tot) {
        if (tid == 0) tile_begin<KIND>(P, sh, sh.ts[0], blockIdx.x);
        __syncthreads();
        if (sh.ts[0].ti.ok && sh.ts[0].ti.nb > 0) setup_lanes<KIND>(P, sh.ts[0]);
        __syncthreads();
    }
    for (int64_t g = blockIdx.x; g < sh.tot; g += gridDim.x, cur ^= PREFETCH ? 1 : 0) {
        TileSetup &ts = sh.ts[cur];
        TileSetup &tn = sh.ts[cur ^ 1];
        const int64_t gn = g + gridDim.x;
        const bool next = PREFETCH && gn < sh.tot;
        if (!PREFETCH) {
            if (tid == 0) tile_begin<KIND>(P, sh, ts, g);
            __syncthreads();
            if (ts.ti.ok && ts.ti.nb > 0) setup_lanes<KIND>(P, ts);
            __syncthreads();
        }
        if (!ts.ti.ok || ts.ti.nb <= 0) {
            if (LIKE && tid == 0) like_store(P, g, 0.0, 0.0);
            if (next) {
                if (tid == 0) tile_begin<KIND>(P, sh, tn, gn);
                __syncthreads();
                if (tn.ti.ok && tn.ti.nb > 0) setup_lanes<KIND>(P, tn);
            }
            __syncthreads();
            continue;
        }
        const int ny = ts.ny, nb = (int)ts.ti.nb;
        double *pf = reinterpret_cast<double *>(smf + OFF_Y);  // raw strain window (FP64)
        // ---- raw strain window and its maximum; TDI-only launches: the link series and the
        //      TDI references
        int wlen = 0;
        long long woff_fx = 0;
        if (KIND != KIND_TDI) {
            const long long span = (long long)ts.whi - (long long)ts.wlo + T + 4;
            const bool wok = span > 0 && span <= MX_WCAP;
            wlen = wok ? (int)span : MX_WCAP;
            if (!wok && tid == 0) atomicOr(P.err, ERR_WINDOW);
            const int woff = wok ? ts.wlo - h - 2 : 0;
            woff_fx = (long long)woff << FX_BITS;
            // the CTA's next tile's bookkeeping (a chain of dependent loads) on the last thread,
            // hidden behind the others' staging loads
            const int nst = next ? MIXED_THREADS - 1 : MIXED_THREADS;
            unsigned long long mx = 0ull;
            if (tid >= nst) {
                tile_begin<KIND>(P, sh, tn, gn);
            } else if (P.gen_strain) {  // the Galactic binary generated at t0 + i dt
                mx = stage_generated(ts.ti.gb, P.t0, P.dt, ts.k_lo + woff, wlen, pf, tid, nst);
            } else {
                for (int j = tid; j < wlen; j += nst) {
                    const int64_t i = ts.k_lo + woff + j;
                    const bool in = i >= 0 && i < ts.ti.nh;
                    const double a = in ? __ldg(ts.ti.hp + i) : 0.0, b = in ? __ldg(ts.ti.hc + i) : 0.0;
                    pf[j] = a;
                    pf[MX_WCAP + j] = b;
                    mx = max(mx, max(abs_bits(a), abs_bits(b)));
                }
            }
            block_absmax(&ts.maxbits, mx);
            __syncthreads();
        } else {
            double *tmp = reinterpret_cast<double *>(smf + OFF_W);
            unsigned long long mx = 0ull;
            for (int l = 0; l < 6; ++l)
                for (int j = tid; j < ny; j += blockDim.x) {
                    const int64_t k = ts.k_lo + j;
                    const double v = (k >= 0 && k < ts.ti.N) ? __ldg(ts.ti.yin + l * ts.ti.N + k) : 0.0;
                    tmp[l * MX_YCAP + j] = v;
                    mx = max(mx, abs_bits(v));
                }
            block_absmax(&ts.maxbits, mx);
            tdi_refs<T>(P, ts, sh, smf + OFF_TW, MIXED_THREADS - NTERM);
            __syncthreads();
        }
        // ---- scaled float-float values
        {
            const int se = tile_scale_exp(ts.maxbits);
            if (tid == 0) {
                sh.unscale_e = -se;
                // a NaN or infinity orders above every finite bit pattern
                if (ts.maxbits >= 0x7ff0000000000000ull) atomicOr(P.err, ERR_NONFINITE);
            }
            if (KIND != KIND_TDI) {
                for (int j = tid; j < wlen; j += blockDim.x) {
                    const ff a = ff_from_double_scaled(pf[j], se), b = ff_from_double_scaled(pf[MX_WCAP + j], se);
                    const int p = phw(j);
                    smf[warr(0, A_SHI) + p] = a.hi;
                    smf[warr(0, A_SLO) + p] = a.lo;
                    smf[warr(1, A_SHI) + p] = b.hi;
                    smf[warr(1, A_SLO) + p] = b.lo;
                }
            } else {
                const double *tmp = reinterpret_cast<const double *>(smf + OFF_W);
                for (int l = 0; l < 6; ++l)
                    for (int j = tid; j < ny; j += blockDim.x) {
                        const ff v = ff_from_double_scaled(tmp[l * MX_YCAP + j], se);
                        smf[ybase(l) + A_SHI * MX_AY + phy(j)] = v.hi;
                        smf[ybase(l) + A_SLO * MX_AY + phy(j)] = v.lo;
                    }
            }
        }
        __syncthreads();
        long long *Lblk = reinterpret_cast<long long *>(smf + OFF_W);
        float *dLf = smf + OFF_W + 2 * 6 * LB;
        if (KIND != KIND_TDI) {
            // ---- strain difference tables
            build_tables2<true, RLW, 4>(smf, warr(0, A_SHI), MX_AW, 7 * MX_AW, 1, wlen);
            __syncthreads();
            // ---- projection reads; then, on the warps with one item: the TDI references and
            //      the next tile's setup
            const int nblk = (ny + PB - 1) / PB;
            for (int it = tid; it < 9 * nblk; it += blockDim.x)
                proj_item<T>(smf, ts, it / nblk, it % nblk, ny, wlen, woff_fx, P.err);
            if (next && tn.ti.ok && tn.ti.nb > 0) setup_lanes<KIND>(P, tn);
            __syncthreads();
            // ---- link series, in place over the staged reads: one thread per sample reads all
            //      of the sample's staged reads before writing its six links (same column)
            for (int j = tid; j < ny; j += blockDim.x) {
                const int ai = phy(j);
                ff rp[3], rc[3];
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    rp[r] = {smf[OFF_Y + (4 * r + 0) * MX_AY + ai], smf[OFF_Y + (4 * r + 1) * MX_AY + ai]};
                    rc[r] = {smf[OFF_Y + (4 * r + 2) * MX_AY + ai], smf[OFF_Y + (4 * r + 3) * MX_AY + ai]};
                }
                const float tau = (float)(j - ts.jc) * TAU_UNIT;
                ff y[6];
                // links in pairs with a common receiving spacecraft r, (0, 3), (1, 5), (2, 4), on
                // the two lanes of packed pairs (each lane the scalar float-float arithmetic)
                const unsigned long long TT = f2pack(tau, tau), TT2 = fmul2(TT, TT);
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    const int l0 = r, l1 = r == 0 ? 3 : (r == 1 ? 5 : 4);
                    auto ld2 = [&](int row) {
                        return f2pack(smf[OFF_Y + (4 * (3 + l0) + row) * MX_AY + ai],
                                      smf[OFF_Y + (4 * (3 + l1) + row) * MX_AY + ai]);
                    };
                    // geometry factor pair at tau: the constant and linear term in float-float (near
                    // a sky direction along an arm 1/(1 - k.n) changes by a large fraction over one
                    // tile), the exact product of the high parts and one two_sum; the low parts,
                    // the product's rounding error and the FP32 quadratic and cubic terms gathered
                    // in the low word (an unnormalised pair, which the product below accepts)
                    auto geom2 = [&](int f0, int f1) {
                        const unsigned long long G1H = f2pack(ts.g1h[f0], ts.g1h[f1]);
                        const unsigned long long Pp = fmul2(G1H, TT);
                        const unsigned long long PE = ffma2(G1H, TT, fneg2(Pp));
                        unsigned long long S, E;
                        two_sum2(f2pack(ts.g0h[f0], ts.g0h[f1]), Pp, S, E);
                        const unsigned long long Q =
                            fmul2(TT2, ffma2(TT, f2pack(ts.g3[f0], ts.g3[f1]), f2pack(ts.g2[f0], ts.g2[f1])));
                        const unsigned long long L =
                            fadd2(E, fadd2(ffma2(f2pack(ts.g1l[f0], ts.g1l[f1]), TT, f2pack(ts.g0l[f0], ts.g0l[f1])),
                                           fadd2(PE, Q)));
                        return ff2{S, L};
                    };
                    const ff2 EP = {ld2(0), ld2(1)}, EC = {ld2(2), ld2(3)};
                    const ff2 RP = {f2pack(rp[r].hi, rp[r].hi), f2pack(rp[r].lo, rp[r].lo)};
                    const ff2 RC = {f2pack(rc[r].hi, rc[r].hi), f2pack(rc[r].lo, rc[r].lo)};
                    const ff2 Y = ff_add2(ff_mul2(geom2(l0, l1), ff_sub2(EP, RP)),
                                          ff_mul2(geom2(6 + l0, 6 + l1), ff_sub2(EC, RC)));
                    f2unpack(Y.hi, y[l0].hi, y[l1].hi);
                    f2unpack(Y.lo, y[l0].lo, y[l1].lo);
                }
                const int64_t k = ts.k_lo + j;
                if (KIND == KIND_PROJECT) {
                    double *o = ts.ti.out;
                    const int64_t N = ts.ti.N;
#pragma unroll
                    for (int l = 0; l < 6; ++l) o[l * N + k] = ff2d_scaled(y[l].hi, y[l].lo, sh.unscale_e);
                } else {
                    const bool in = k >= 0 && k < ts.ti.N;
#pragma unroll
                    for (int l = 0; l < 6; ++l) {
                        smf[ybase(l) + A_SHI * MX_AY + ai] = in ? y[l].hi : 0.0f;
                        smf[ybase(l) + A_SLO * MX_AY + ai] = in ? y[l].lo : 0.0f;
                    }
                }
            }
            // the TDI references of this tile, on threads that the loop above gave one sample
            if (FUSED) tdi_refs<T>(P, ts, sh, smf + OFF_TW, TDI_REF0);
        }
        double *ld = reinterpret_cast<double *>(smf + OFF_LD);
        if (KIND != KIND_PROJECT) {
            // likelihood launches: the tile's A, E, T data, fetched asynchronously for the
            // epilogue (the strain tables are no longer read)
            if (LIKE && ts.ti.dat) {
                const double *src = ts.ti.dat + ts.ti.n0;
                for (int j = tid; j < 3 * nb; j += blockDim.x) {
                    const int c = j / nb, i = j - c * nb;
                    cp_async8(ld + c * XYZ_CAP + i, src + c * ts.ti.N + i);
                }
            }
            // link delays of the outputs: at each item's first output (fixed point) and the
            // increments to the item's other outputs (rows padded to whole items)
            static_assert(TB == 4, "one float4 of increments per TDI item");
            const int nbt = (nb + TB - 1) / TB;
            for (int idx = tid; idx < 6 * nbt; idx += blockDim.x) {
                const int l = idx / nbt, bi = idx - l * nbt, i0 = TB * bi;
                const long long L0 = piece_at(ts.dp[i0 < ts.jswt ? 0 : 1][l], i0 - ts.ic);
                Lblk[l * LB + bi] = L0;
                float d[TB];
                d[0] = 0.0f;
#pragma unroll
                for (int k = 1; k < TB; ++k) {
                    const int i = i0 + k;
                    d[k] = (float)(piece_at(ts.dp[i < ts.jswt ? 0 : 1][l], i - ts.ic) - L0);
                }
                reinterpret_cast<float4 *>(dLf + l * LT)[bi] = make_float4(d[0], d[1], d[2], d[3]);
            }
            __syncthreads();
            // ---- link difference tables
            build_tables2<false, RLY, 5>(smf, ybase(0), MX_AY, 6 * MX_AY, 3, ny);
            __syncthreads();
            // ---- X, Y, Z
            const int nbb = (nb + TB - 1) / TB;
            for (int it = tid; it < 3 * nbb; it += blockDim.x) {
                const int ch = it / nbb, b = it - ch * nbb, i0 = TB * b;
                const int kmax = min(TB, nb - i0);
                // float-float accumulators (hi, lo) and the FP32 small terms, packed over output pairs
                unsigned long long HI[TB / 2], LO[TB / 2], SM[TB / 2];
#pragma unroll
                for (int pr = 0; pr < TB / 2; ++pr) HI[pr] = LO[pr] = SM[pr] = 0ull;
                // X = A - B = -((-A) + B): both chains through one code copy
#pragma unroll 1
                for (int c = 0; c < 2; ++c) {
                    tdi_chain<T>(P, sh, ny, smf, Lblk, dLf, ch, c, b, kmax, HI, LO, SM);
#pragma unroll
                    for (int pr = 0; pr < TB / 2; ++pr) {
                        HI[pr] = fneg2(HI[pr]);
                        LO[pr] = fneg2(LO[pr]);
                        SM[pr] = fneg2(SM[pr]);
                    }
                }
                // X, Y, Z to global memory (likelihood launches: only when asked for) and, for the
                // likelihood epilogue, as scaled FP32 values on chip
                double *o = !LIKE || ts.ti.out ? ts.ti.out + ch * ts.ti.N + ts.ti.n0 + i0 : nullptr;
                float *xs = LIKE ? smf + OFF_XYZ + ch * XYZ_CAP + i0 : nullptr;
#pragma unroll
                for (int k = 0; k < TB; ++k)
                    if (k < kmax) {
                        const float hi = lane(HI[k >> 1], k & 1), lo = lane(LO[k >> 1], k & 1) + lane(SM[k >> 1], k & 1);
                        if (!LIKE || o) o[k] = ff2d_scaled(hi, lo, sh.unscale_e);
                        if (LIKE) xs[k] = hi + lo;
                    }
            }
            // ---- likelihood epilogue: A, E, T of the tile against the data, block sums
            if (LIKE) {
                cp_async_wait_all();
                __syncthreads();
                const int se = -sh.unscale_e;
                const float *xs = smf + OFF_XYZ;
                float dh = 0.0f, hh = 0.0f;
                bool bad = false;
                if (ts.ti.dat)
                    for (int i = tid; i < nb; i += blockDim.x) {
                        bad |= !(isfinite(ld[i]) && isfinite(ld[XYZ_CAP + i]) && isfinite(ld[2 * XYZ_CAP + i]));
                        like_terms_f(P.like, xs[i], xs[XYZ_CAP + i], xs[2 * XYZ_CAP + i],
                                     ff_from_double_scaled(ld[i], se).hi, ff_from_double_scaled(ld[XYZ_CAP + i], se).hi,
                                     ff_from_double_scaled(ld[2 * XYZ_CAP + i], se).hi, dh, hh);
                    }
                if (bad) atomicOr(P.err, ERR_NONFINITE);
                block_sum2f(dh, hh, sh.redf);
                // undo the scale 2^se of both factors (exactly, by integer work); the weight
                // normalisation is undone once per source by the reduction
                if (tid == 0)
                    like_store(P, g, ts.ti.dat ? f2d_pow2(dh, -2 * se) : nan_d(),
                               ts.ti.dat ? f2d_pow2(hh, -2 * se) : nan_d());
            }
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace lr
