// Launch layer: picks the kernel family for a plan's precision and sizes the persistent grid.
#pragma once
#include "lr_internal.h"

namespace lr {
bool order_supported(int order);
bool precision_supported(int precision);
int default_tile(int precision, int order);
// returns a cudaError_t value (0 = success)
int launch_forward(int precision, int kind, int order, FwdParams &P, int threads, int sms, void *stream);
int launch_tile_offsets(const int64_t *out_off, int64_t S, int tile, int64_t *tile_off, int *err, void *stream);
// tile table and, when skyc is not null, the sky frame of every source
int launch_batch_tables(const int64_t *out_off, const lr_sky *sky, int64_t S, int tile, int64_t *tile_off,
                        SkyConst *skyc, int *err, void *stream);
bool order_compiled(int order);
// g = scale * d(<d|h> - <h|h>/2)/d(X, Y, Z) per sample; the arrays hold n1 samples per channel
// block (out_off == nullptr: one source of n1)
int launch_like_grad(const int64_t *out_off, int64_t S, int64_t n1, const double *x, const double *d,
                     const double *w, double scale, double *g, int *err, void *stream);
// per-source (<d|h>, <h|h>) from the per-tile partials of a likelihood launch, times post; with
// logl != 0 one value per source instead, <d|h> - <h|h>/2
int launch_like_reduce(const double *partial, const int64_t *tile_off, int64_t tiles1, int64_t S, int64_t cap,
                       double post, int logl, double *out, int *err, void *stream);
}  // namespace lr
