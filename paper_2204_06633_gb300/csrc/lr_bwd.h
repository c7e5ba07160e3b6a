// Backward launch parameters shared by the host and the adjoint kernels.
#pragma once
#include "lr_internal.h"

namespace lr {

struct BwdParams {
    const double *g_xyz;        // [3][n] per source (same offsets as the outputs)
    double *g_y;                // [6][n] per source (plan-owned workspace)
    double *g_hp, *g_hc;        // [n_h] per source (same offsets as the inputs)
    double *partial;            // [tiles][3] per-tile sky-gradient partial sums (workspace)
    const int64_t *h_tile_off;  // [S+1] strain-tile prefix sums (batched) or nullptr
    int64_t h_total_tiles;      // >= 0 single source; -1: read h_tile_off[S]
    int tile_h;                 // strain samples per transpose-of-projection tile
    int wn;                     // capacity of the TDI-transpose output window
    int wk;                     // capacity of the projection-transpose link window
    int dmax;                   // bound of chained delays, samples
    int kmargin;                // link-window margin for the drift of read times over a tile
};

constexpr int BWD_TILE_K = 256;  // link samples per TDI-transpose / sky tile (= threads)
constexpr int BWD_TILE_H = 128;  // strain samples per projection-transpose tile

// kind 0: TDI transpose, 1: projection transpose, 2: sky-gradient partials
int launch_bwd(int kind, int order, const FwdParams &P, const BwdParams &B, int sms, void *stream);
size_t smem_bwd(int kind, int order, const FwdParams &P, const BwdParams &B);
// mixed-precision adjoint kernels for plans of precision LR_MIXED (kind 0: TDI transpose, 1:
// projection transpose, 2: sky-gradient partials)
int launch_bwd_mx(int kind, int order, const FwdParams &P, const BwdParams &B, int sms, void *stream);
size_t smem_bwd_mx(int kind, int order, const FwdParams &P, const BwdParams &B);
int launch_sky_reduce(const double *partial, const int64_t *tile_off, int64_t S, int64_t ntiles1, double *g_sky,
                      void *stream);

}  // namespace lr
