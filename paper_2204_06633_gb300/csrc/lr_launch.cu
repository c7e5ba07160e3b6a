// Launch layer: kernel-family dispatch, persistent grid sizing and the batch tile table.
#include <cuda_runtime.h>

#include "lr_launch.h"

namespace lr {

bool order_supported(int order) { return order >= 1 && (order & 1) && order_compiled(order) && order_compiled_mx(order); }

bool precision_supported(int precision) { return precision == LR_FP64 || precision == LR_MIXED; }

int default_tile(int precision, int order)
{
    (void)order;
    return precision == LR_MIXED ? 256 : 512;
}

int launch_forward(int precision, int kind, int order, FwdParams &P, int threads, int sms, void *stream)
{
    const bool mx = precision == LR_MIXED;
    if (mx) threads = MIXED_THREADS;
    size_t smem = 0;
    if (mx) smem_fwdmx(kind, order, P, &smem); else smem_fwd64(kind, order, P, &smem);
    int per_sm = 0;
    int e = mx ? max_blocks_fwdmx(kind, order, threads, smem, &per_sm) : max_blocks_fwd64(kind, order, threads, smem, &per_sm);
    if (e) return e;
    if (per_sm < 1) return (int)cudaErrorLaunchOutOfResources;
    int64_t grid = (int64_t)per_sm * sms;
    if (P.total_tiles >= 0 && P.total_tiles < grid) grid = P.total_tiles;
    if (grid < 1) grid = 1;
    return mx ? launch_fwdmx(kind, order, P, (int)grid, threads, smem, stream)
              : launch_fwd64(kind, order, P, (int)grid, threads, smem, stream);
}

// Prefix sums of tiles per source (one block; each thread scans a contiguous chunk of
// sources, then the chunk totals are scanned in shared memory).  Decreasing offsets are
// recorded as ERR_OFFSETS and count as empty sources.
__global__ void __launch_bounds__(1024) k_tile_offsets(const int64_t *__restrict__ out_off, int64_t S, int tile,
                                                       int64_t *__restrict__ tile_off, int *err)
{
    __shared__ int64_t part[1024];
    const int64_t chunk = (S + blockDim.x - 1) / blockDim.x;
    const int64_t s0 = threadIdx.x * chunk;
    const int64_t s1 = s0 + chunk < S ? s0 + chunk : S;
    int64_t sum = 0;
    for (int64_t s = s0; s < s1; ++s) {
        int64_t n = out_off[s + 1] - out_off[s];
        if (n < 0) {
            atomicOr(err, ERR_OFFSETS);
            n = 0;
        }
        sum += (n + tile - 1) / tile;
    }
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        int64_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = part[threadIdx.x] - sum;  // exclusive prefix of this chunk
    for (int64_t s = s0; s < s1; ++s) {
        tile_off[s] = run;
        int64_t n = out_off[s + 1] - out_off[s];
        if (n < 0) n = 0;
        run += (n + tile - 1) / tile;
    }
    if (threadIdx.x == blockDim.x - 1) tile_off[S] = part[threadIdx.x];
}

int launch_tile_offsets(const int64_t *out_off, int64_t S, int tile, int64_t *tile_off, int *err, void *stream)
{
    k_tile_offsets<<<1, 1024, 0, (cudaStream_t)stream>>>(out_off, S, tile, tile_off, err);
    return (int)cudaGetLastError();
}

__global__ void k_sky_consts(const lr_sky *__restrict__ sky, int64_t S, SkyConst *__restrict__ out)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x)
        out[s] = make_sky(sky[s]);
}

int launch_batch_tables(const int64_t *out_off, const lr_sky *sky, int64_t S, int tile, int64_t *tile_off,
                        SkyConst *skyc, int *err, void *stream)
{
    int e = launch_tile_offsets(out_off, S, tile, tile_off, err, stream);
    if (e || !skyc) return e;
    const int64_t blocks = (S + 255) / 256;
    k_sky_consts<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, (cudaStream_t)stream>>>(sky, S, skyc);
    return (int)cudaGetLastError();
}

// Per-source sums of the likelihood partials: one warp per source adds its tiles' partials
// (lane l takes tiles l, l + 32, ... in order, then a fixed shuffle tree), so the result does not
// depend on the launch or on timing; the sums are multiplied by post (the weight normalisation
// of the mixed epilogue, 1 otherwise).  tile_off == nullptr: one source of tiles1 tiles.
// logl != 0: out[s] = (<d|h> - <h|h>/2) * post instead of the pair.
__global__ void __launch_bounds__(256) k_like_reduce(const double *__restrict__ partial,
                                                     const int64_t *__restrict__ tile_off, int64_t tiles1,
                                                     int64_t S, int64_t cap, double post, int logl,
                                                     double *__restrict__ out, int *err)
{
    const int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (s >= S) return;  // uniform over the warp
    const int64_t a = tile_off ? tile_off[s] : 0, b = tile_off ? tile_off[s + 1] : tiles1;
    if (a < 0 || b < a || b > cap) {
        if (lane == 0) {
            atomicOr(err, ERR_OFFSETS);
            const double nan = __longlong_as_double(0x7ff8000000000000ll);
            if (logl) out[s] = nan;
            else out[2 * s] = out[2 * s + 1] = nan;
        }
        return;
    }
    double dh = 0.0, hh = 0.0;
    for (int64_t g = a + lane; g < b; g += 32) {
        dh += partial[2 * g];
        hh += partial[2 * g + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        dh += __shfl_down_sync(0xffffffffu, dh, o);
        hh += __shfl_down_sync(0xffffffffu, hh, o);
    }
    if (lane == 0) {
        if (logl) {
            out[s] = fma(-0.5, hh, dh) * post;
        } else {
            out[2 * s] = dh * post;
            out[2 * s + 1] = hh * post;
        }
    }
}

// Gradient of the time-domain log-likelihood <d|h> - <h|h>/2 (A, E, T channels, weights w) with
// respect to the template's X, Y, Z: g = scale * M^T W (d - M x), M the A, E, T map (rows
// (-1, 0, 1)/sqrt 2, (1, -2, 1)/sqrt 6, (1, 1, 1)/sqrt 3).  Source s (of S) holds [3][N_s] at
// 3 out_off[s] in x, d and g, which hold n1 samples per channel block (sources past them are
// skipped and recorded); out_off == nullptr: one source of n1 samples.  Blocks walk sources,
// threads walk samples.
__global__ void __launch_bounds__(256) k_like_grad(const int64_t *__restrict__ out_off, int64_t S, int64_t n1,
                                                   const double *__restrict__ x, const double *__restrict__ d,
                                                   double w0, double w1, double w2, double scale,
                                                   double *__restrict__ g, int *err)
{
    const double R2 = 0.70710678118654752440, R6 = 0.40824829046386301637, R3 = 0.57735026918962576451;
    for (int64_t s = blockIdx.x; s < S; s += gridDim.x) {
        const int64_t o = out_off ? out_off[s] : 0, N = out_off ? out_off[s + 1] - o : n1;
        if (N < 0 || o < 0 || o + N > n1) {
            if (threadIdx.x == 0) atomicOr(err, ERR_OFFSETS);
            continue;
        }
        const double *xs = x + 3 * o, *ds = d + 3 * o;
        double *gs = g + 3 * o;
        for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
            const double X = xs[i], Y = xs[N + i], Z = xs[2 * N + i];
            const double s2 = X + Z;
            const double ra = w0 * (ds[i] - (Z - X) * R2), re = w1 * (ds[N + i] - fma(-2.0, Y, s2) * R6),
                         rt = w2 * (ds[2 * N + i] - (s2 + Y) * R3);
            const double e6 = re * R6, t3 = rt * R3;
            gs[i] = scale * (fma(-ra, R2, e6) + t3);
            gs[N + i] = scale * fma(-2.0, e6, t3);
            gs[2 * N + i] = scale * (fma(ra, R2, e6) + t3);
        }
    }
}

int launch_like_grad(const int64_t *out_off, int64_t S, int64_t n1, const double *x, const double *d,
                     const double *w, double scale, double *g, int *err, void *stream)
{
    const int64_t blocks = S < 4096 ? S : 4096;
    k_like_grad<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(out_off, S, n1, x, d, w[0], w[1], w[2], scale, g,
                                                                   err);
    return (int)cudaGetLastError();
}

int launch_like_reduce(const double *partial, const int64_t *tile_off, int64_t tiles1, int64_t S, int64_t cap,
                       double post, int logl, double *out, int *err, void *stream)
{
    const int64_t blocks = (S + 7) / 8;
    k_like_reduce<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(partial, tile_off, tiles1, S, cap, post, logl,
                                                                     out, err);
    return (int)cudaGetLastError();
}

}  // namespace lr
