// Internal types shared by the host side of the library and its kernels.
#pragma once
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

// Per-call description of the sources processed by a launch.
struct SrcArgs {
    // batched: device arrays (nullptr for a single-source launch)
    const int64_t *h_off;
    const int64_t *out_off;
    const double *t0h;
    const lr_sky *sky;
    const int64_t *tile_off;  // [S+1] prefix sums of tiles per source
    int64_t S;
    // single source
    int64_t n1, nh1;
    double t0h1;
    lr_sky sky1;
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
    const double *yin;      // link series input (TDI-only launches)
    double *out;            // y [6][n] or xyz [3][n]
    int *err;               // device error word
    int64_t total_tiles;    // >= 0 single source; -1: read src.tile_off[S]
    double cheb[4][4];      // monomial coefficients of the cubic through 4 Chebyshev nodes on [-1, 1]
};

// error-word bits
constexpr int ERR_WINDOW = 1;    // a stencil fell outside its staged window
constexpr int ERR_OFFSETS = 2;   // batched offsets not monotone
constexpr int ERR_TIMEOUT = 4;   // bounded wait ran out

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
enum { KIND_PROJECT = 0, KIND_TDI = 1, KIND_FUSED = 2 };
}  // namespace lr
