// Internal types shared by the host side of the library and its kernels.
#pragma once
#include <math.h>
#include <stdint.h>

#include "lisaresp.h"

namespace lr {

constexpr double C_LIGHT = 299792458.0;
constexpr int NSERIES = 15;   // x1 y1 z1 x2 y2 z2 x3 y3 z3, L12 L23 L31 L13 L32 L21
constexpr int MAX_TAPS = 64;  // order 63
constexpr int CHAIN_TERMS = 8;  // terms per Michelson chain (q = 0 undelayed .. 7)

// Cubic-spline tables of one orbit on a uniform knot grid: on interval k and for series s the
// value is a + x (b + x (c + x d)) with x = (t - t_first)/dk - k (x in [0,1) inside the grid;
// the end pieces are continued outside it).
struct OrbitDev {
    const double *coef;  // [nint][NSERIES][4]
    int nint;
    double t_first;
    double inv_dk;
};

// TDI chain tables.  Each Michelson combination is two chains of the form
//   sign * sum_{q=0..Q} D_{c_0 .. c_q} y_{c_q c_{q+1}}
// (Q = 3 for the first generation, 7 for the second): chain A (+) of X runs over the
// spacecraft sequence 1 3 1 2 1 2 1 3 1 and chain B (-) over 1 2 1 3 1 3 1 2 1 (Eqs. tdi1,
// tdi2); Y and Z apply the cyclic map 1->2->3->1.  link[q] is the series read by term q and
// pair[q] (q >= 1) the link whose delay is added when going from term q-1 to term q.
struct TdiTab {
    signed char link[3][2][CHAIN_TERMS];
    signed char pair[3][2][CHAIN_TERMS];
};

// Sky frame of a source: k = -e_r, u = -e_phi, v = -e_theta of the SSB basis (Sec. "Reference
// frames"); c2p, s2p rotate the antenna patterns by 2 psi.
struct SkyConst {
    double k[3], u[3], v[3];
    double c2p, s2p;
};

__host__ __device__ inline SkyConst make_sky(const lr_sky &s)
{
    SkyConst c;
    double sl, cl, sb, cb, s2, c2;
#ifdef __CUDA_ARCH__
    sincos(s.lam, &sl, &cl);
    sincos(s.beta, &sb, &cb);
    sincos(2.0 * s.psi, &s2, &c2);
#else
    sl = sin(s.lam); cl = cos(s.lam);
    sb = sin(s.beta); cb = cos(s.beta);
    s2 = sin(2.0 * s.psi); c2 = cos(2.0 * s.psi);
#endif
    c.k[0] = -cb * cl; c.k[1] = -cb * sl; c.k[2] = -sb;
    c.u[0] = sl;       c.u[1] = -cl;      c.u[2] = 0.0;
    c.v[0] = -sb * cl; c.v[1] = -sb * sl; c.v[2] = cb;
    c.c2p = c2; c.s2p = s2;
    return c;
}

// Per-call description of the sources processed by a launch.
struct SrcArgs {
    // batched: device arrays (nullptr for a single-source launch)
    const int64_t *h_off;
    const int64_t *out_off;
    const double *t0h;
    const lr_sky *sky;
    const int64_t *tile_off;  // [S+1] prefix sums of tiles per source
    const SkyConst *skyc;     // [S] sky frames (mixed launches; nullptr otherwise)
    int64_t S;
    // single source
    int64_t n1, nh1;
    double t0h1;
    lr_sky sky1;
    SkyConst skyc1;
    // strain generated on the device (FwdParams::gen_strain): Galactic-binary parameters, device
    // [S] (batched) or gb1 (single source)
    const lr_gb *gb;
    lr_gb gb1;
};

// Fused likelihood epilogue of the forward launch (Eq. like in the time domain, summed over the
// channels A, E, T of Sec. "Time-delay interferometry"): each tile leaves its partial
// (<d|h>, <h|h>) in partial[2 g], [2 g + 1]; a second kernel sums the tiles of every source in
// a fixed order.  data == nullptr: no likelihood.
struct LikeArgs {
    const double *data;  // data in A, E, T: [3][N_s] per source, at 3 out_off[s] (batched)
    double w[3];         // channel weights (1 / noise variance of A, E, T)
    double wmax;         // largest weight; wn = w / wmax in FP32 (mixed epilogue)
    float wn[3];
    double *partial;     // [cap][2]
    int64_t cap;         // tiles the partial buffer holds
    int64_t n_total;     // samples the data array holds per channel block (sum of N_s)
};

struct FwdParams {
    double dt, inv_dt, t0;
    OrbitDev po, to;      // projection orbit, TDI orbit
    TdiTab tdi;
    int q_terms;          // 3 (generation 1) or 7 (generation 2)
    int delay_nested;     // 0 summed, 1 nested
    int tile;             // outputs per tile
    int HL, HR;           // link-series halo of a tile (samples)
    int sig_b;            // bound of |k.x|/(c dt) over the orbit, samples
    int lproj_b;          // bound of projection delays / dt, samples
    int wmax;             // capacity of the staged strain window
    int ymax;             // capacity of the staged link window (tile + HL + HR)
    SrcArgs src;
    const double *hp, *hc;  // strain (h+, hx)
    int gen_strain;         // 1: the strain is a Galactic binary generated on the device (src.gb),
                            // sampled on the output grid t0 + i dt at every i (no zero extension)
    const double *yin;      // link series input (TDI-only launches)
    double *out;            // y [6][n] or xyz [3][n] (fused likelihood launches: may be null)
    LikeArgs like;
    int *err;               // device error word
    int64_t total_tiles;    // >= 0 single source; -1: read src.tile_off[S]
    // nested chained delays in the mixed kernels: per delayed term (42) the nested minus the
    // summed total delay (samples) at the TDI orbit's knots, interpolated linearly per tile;
    // null for summed delays
    const double *nest_tab;  // [nest_n][42]
    int nest_n;
    double nest_t0, nest_inv_dk;
    double cheb[4][4];      // monomial coefficients of the cubic through 4 Chebyshev nodes on [-1, 1]
    double cheb_node[4];    // the nodes cos((2 i + 1) pi / 8)
    // constant TDI delays (every delay spline of the TDI orbit constant): per delayed term
    // (channel, chain, q = 1..7) the Lagrange weights of its fixed fractional offset,
    // [3][2][8][T] FP64 (q = 0 unused), and the first tap's offset from the output sample;
    // null when the delays vary (FP64 kernels only)
    const double *cd_w;
    int cd_off[3][2][CHAIN_TERMS];
};

// generated strain: the source's waveform sampled on the output grid at every index (the
// strain length used in the window bounds)
constexpr int64_t GEN_STRAIN_LEN = (int64_t)1 << 62;

// error-word bits
constexpr int ERR_WINDOW = 1;    // a stencil fell outside its staged window
constexpr int ERR_OFFSETS = 2;   // batched offsets not monotone
constexpr int ERR_TIMEOUT = 4;   // bounded wait ran out
constexpr int ERR_NONFINITE = 8; // a NaN or infinity in the strain or likelihood data a tile read

}  // namespace lr

// kernel launchers (one translation unit per precision family)
namespace lr {
int launch_fwd64(int kind, int order, const FwdParams &P, int grid, int threads, size_t smem, void *stream);
int smem_fwd64(int kind, int order, const FwdParams &P, size_t *smem);
int max_blocks_fwd64(int kind, int order, int threads, size_t smem, int *blocks);
int launch_fwdmx(int kind, int order, const FwdParams &P, int grid, int threads, size_t smem, void *stream);
int smem_fwdmx(int kind, int order, const FwdParams &P, size_t *smem);
int max_blocks_fwdmx(int kind, int order, int threads, size_t smem, int *blocks);
bool order_compiled_mx(int order);
constexpr int MIXED_THREADS = 256;  // the mixed kernels' per-tile setup assigns work by thread index

// Shared-memory geometry of the mixed kernels (compile time, so every array offset is an
// immediate).  A staged series of up to n samples is stored in 8 phases: sample j at
// (j mod 8) * RL + j / 8, with the row length RL four times an odd number; consecutive
// samples, and every 4th or 8th sample across a warp, then fall in distinct banks.
constexpr int MX_YCAP = 384;  // link span of a tile (outputs + TDI halo)
constexpr int MX_WCAP = 466;  // strain window of a tile
__host__ __device__ constexpr int mx_rl(int n) { return ((((n + 7) / 8 + 3) & ~3) / 4) % 2 ? (((n + 7) / 8 + 3) & ~3) : (((n + 7) / 8 + 3) & ~3) + 4; }
constexpr int MX_AY = 8 * mx_rl(MX_YCAP);  // floats per link-span array
constexpr int MX_AW = 8 * mx_rl(MX_WCAP);  // floats per strain-window array
constexpr int MX_TDI_BLOCK = 4;            // consecutive outputs per TDI work item
// correction-weight pairs (U, dU/deps) per TDI term, padded to a multiple of 2 pairs
__host__ __device__ constexpr int mx_nup(int T) { return T >= 4 ? ((T - 3 + 1) & ~1) : 2; }
// strain tables, link tables, TDI weights
__host__ __device__ constexpr int mx_smem_floats(int T) { return 14 * MX_AW + 36 * MX_AY + 42 * 2 * mx_nup(T); }
// largest tile the mixed kernels stage: the link span within MX_YCAP, the strain window
// (span + read spread 2 lproj_b + T + 6) within MX_WCAP, TDI items (3 channels x tile/4) in
// one pass of the threads
inline int mx_max_tile(int HL, int HR, int lproj_b, int T)
{
    int t = MX_YCAP - HL - HR;
    int w = MX_WCAP - 2 * lproj_b - T - 6 - HL - HR;
    if (w < t) t = w;
    int one_pass = MX_TDI_BLOCK * (MIXED_THREADS / 3);
    if (one_pass < t) t = one_pass;
    return t & ~(MX_TDI_BLOCK - 1);
}
// launch kinds: projection only, TDI only, fused, fused with the likelihood epilogue
enum { KIND_PROJECT = 0, KIND_TDI = 1, KIND_FUSED = 2, KIND_LIKE = 3 };
}  // namespace lr
