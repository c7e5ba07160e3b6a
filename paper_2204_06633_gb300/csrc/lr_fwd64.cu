// FP64 forward kernels: projection onto the six links, TDI, and the fused projection+TDI.
//
// Work unit: a tile of `tile` consecutive output samples of one source.  A CTA stages the
// strain window its tile reads (all read times of the tile: global light-time shift
// |k.x|/c <= sig_b samples, emitter delay <= lproj_b samples, stencil) in shared memory,
// computes the link series for the tile plus the TDI halo into shared memory, and forms
// X, Y, Z from there; CTAs loop over tiles (persistent grid sized to the SM count).
#include <cuda_runtime.h>

#include "lr_device.cuh"
#include "lr_tdi_table.cuh"

namespace lr {

__constant__ TdiTab c_tdi64 = make_tdi_tab();

// ---------------------------------------------------------------- projection of one sample
// y_l(t_k) = [H_l(t - L_l - k.x_s/c) - H_l(t - k.x_r/c)] / (2 (1 - k.n_l))   (Eq.
// instrument-response-to-gw), H_l = xi+_l h+ + xix_l hx with the patterns rotated by 2 psi.
// Read positions in the strain grid are k + u with u = (t0 - t0_h)/dt - (shift)/dt.
template <int T>
__device__ void project_sample64(const FwdParams &P, const SkyConst &S, int64_t k, double u0,
                                 const double *hwp, const double *hwc, int64_t w_lo, int wlen, double y[6])
{
    double t = P.t0 + (double)k * P.dt;
    double x[9], L[6];
    orbit_all(P.po, t, x, L);
    double sig[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        sig[i] = (S.k[0] * x[3 * i] + S.k[1] * x[3 * i + 1] + S.k[2] * x[3 * i + 2]) / C_LIGHT * P.inv_dt;
    double rp[3], rc[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) read2<T>(hwp, hwc, k, u0 - sig[i], w_lo, wlen, rp[i], rc[i], P.err);
    // arms 12, 23, 31 (links 0, 1, 2) and their reverses 21, 32, 13 (links 5, 4, 3)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int r = a, s = (a + 1) % 3;
        const int lf = a, lr_ = 5 - a;
        double d0 = x[3 * r] - x[3 * s], d1 = x[3 * r + 1] - x[3 * s + 1], d2 = x[3 * r + 2] - x[3 * s + 2];
        double inv = 1.0 / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        d0 *= inv; d1 *= inv; d2 *= inv;
        double un = S.u[0] * d0 + S.u[1] * d1 + S.u[2] * d2;
        double vn = S.v[0] * d0 + S.v[1] * d1 + S.v[2] * d2;
        double kn = S.k[0] * d0 + S.k[1] * d1 + S.k[2] * d2;
        double xip = un * un - vn * vn, xic = 2.0 * un * vn;
        double xp = S.c2p * xip + S.s2p * xic, xc = -S.s2p * xip + S.c2p * xic;
        double ep, ec;
        read2<T>(hwp, hwc, k, u0 - L[lf] * P.inv_dt - sig[s], w_lo, wlen, ep, ec, P.err);
        y[lf] = (xp * (ep - rp[r]) + xc * (ec - rc[r])) / (2.0 * (1.0 - kn));
        read2<T>(hwp, hwc, k, u0 - L[lr_] * P.inv_dt - sig[r], w_lo, wlen, ep, ec, P.err);
        y[lr_] = (xp * (ep - rp[s]) + xc * (ec - rc[s])) / (2.0 * (1.0 + kn));
    }
}

// ---------------------------------------------------------------- TDI of one sample
// X = sum_q D_{chain A up to q} y_link(A,q) - sum_q D_{chain B up to q} y_link(B,q); the
// delay of term q is the sum (or nesting) of the chain's first q link delays, all at t_n.
// Constant delays: every delayed read of a term has the same fractional offset, so its weights
// are plan constants and a read is a plain T-tap dot product.
template <int T>
__device__ void tdi_sample64_const(const FwdParams &P, int64_t n, const double *ys, int ystride, int64_t k_lo,
                                   int ylen, double out[3])
{
    const int nl = (int)(n - k_lo);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            double part = ys[c_tdi64.link[ch][c][0] * ystride + nl];
            for (int q = 1; q <= P.q_terms; ++q) {
                const int st = nl + P.cd_off[ch][c][q];
                if (st < 0 || st + T > ylen) {
                    atomicOr(P.err, ERR_WINDOW);
                    continue;
                }
                const double *s = ys + c_tdi64.link[ch][c][q] * ystride + st;
                const double *w = P.cd_w + ((ch * 2 + c) * CHAIN_TERMS + q) * T;
                double r = 0.0;
#pragma unroll
                for (int j = 0; j < T; ++j) r = fma(__ldg(w + j), s[j], r);
                part += r;
            }
            acc = c == 0 ? part : acc - part;
        }
        out[ch] = acc;
    }
}

template <int T>
__device__ void tdi_sample64(const FwdParams &P, int64_t n, const double *ys, int ystride, int64_t k_lo,
                             int ylen, double out[3])
{
    if (P.cd_w) {
        tdi_sample64_const<T>(P, n, ys, ystride, k_lo, ylen, out);
        return;
    }
    double t = P.t0 + (double)n * P.dt;
    double Ls[6];
    orbit_delays(P.to, t, Ls);
#pragma unroll
    for (int l = 0; l < 6; ++l) Ls[l] *= P.inv_dt;
    const int nl = (int)(n - k_lo);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            double part = ys[c_tdi64.link[ch][c][0] * ystride + nl];
            double D = 0.0;
            for (int q = 1; q <= P.q_terms; ++q) {
                int pr = c_tdi64.pair[ch][c][q];
                double u;
                if (P.delay_nested) {
                    D += orbit_delay1(P.to, t - D, pr);   // seconds
                    u = -D * P.inv_dt;
                } else {
                    D += Ls[pr];                           // samples
                    u = -D;
                }
                part += read1<T>(ys + c_tdi64.link[ch][c][q] * ystride, n, u, k_lo, ylen, P.err);
            }
            acc = c == 0 ? part : acc - part;
        }
        out[ch] = acc;
    }
}

// strain window of a tile whose link samples cover [k_lo, k_lo + ny)
__device__ inline void strain_window(const FwdParams &P, int T, int64_t k_lo, int ny, double u0, int64_t *w_lo,
                                     int *wlen)
{
    const int h = (T - 2) / 2;
    *w_lo = k_lo + (int64_t)floor(u0) - P.sig_b - P.lproj_b - h - 2;
    *wlen = ny + 2 * P.sig_b + P.lproj_b + T + 4;
}

__device__ inline void stage(double *dst, const double *src, int64_t lo, int len, int64_t n_src)
{
    for (int j = threadIdx.x; j < len; j += blockDim.x) {
        int64_t i = lo + j;
        dst[j] = (i >= 0 && i < n_src) ? __ldg(src + i) : 0.0;
    }
}

// stage() of the strain, recording a NaN or infinity in the error word
__device__ inline void stage_checked(double *dst, const double *src, int64_t lo, int len, int64_t n_src, int *err)
{
    bool bad = false;
    for (int j = threadIdx.x; j < len; j += blockDim.x) {
        int64_t i = lo + j;
        const double v = (i >= 0 && i < n_src) ? __ldg(src + i) : 0.0;
        dst[j] = v;
        bad |= !isfinite(v);
    }
    if (bad) atomicOr(err, ERR_NONFINITE);
}

// generated strain window (out of line: keeps the sincos out of the hot body)
__device__ __noinline__ void stage_generated64(const GbConst &g, double t0, double dt, int64_t lo, int len, double *hwp,
                                               double *hwc)
{
    for (int j = threadIdx.x; j < len; j += blockDim.x) gb_strain(g, t0, dt, lo + j, hwp[j], hwc[j]);
}

// the strain window of a tile: staged from the caller's arrays, or generated (Galactic binary on
// the output grid, strain index = output index)
__device__ inline void stage_strain(const FwdParams &P, const TileInfo &ti, double *hwp, double *hwc, int64_t lo,
                                    int len)
{
    if (P.gen_strain) {
        stage_generated64(ti.gb, P.t0, P.dt, lo, len, hwp, hwc);
    } else {
        stage_checked(hwp, ti.hp, lo, len, ti.nh, P.err);
        stage_checked(hwc, ti.hc, lo, len, ti.nh, P.err);
    }
}

// ---------------------------------------------------------------- kernels
template <int T>
__global__ void __launch_bounds__(256, 2) k_fused64(FwdParams P)
{
    extern __shared__ double sm[];
    double *hwp = sm, *hwc = sm + P.wmax, *ys = sm + 2 * P.wmax;
    __shared__ TileInfo ti;
    __shared__ SkyConst skc;
    __shared__ double red[2 * 32];
    const bool like = P.like.data != nullptr;
    const int64_t total = P.total_tiles >= 0 ? P.total_tiles : P.src.tile_off[P.src.S];
    for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
        if (threadIdx.x == 0) {
            ti = tile_info(P, g, 3);
            skc = make_sky(ti.sky);
            if (!ti.ok) atomicOr(P.err, ERR_OFFSETS);
            if (like && !(ti.ok && ti.nb > 0)) like_store(P, g, 0.0, 0.0);
        }
        __syncthreads();
        if (ti.ok && ti.nb > 0) {
            const int64_t k_lo = ti.n0 - P.HL;
            const int ny = (int)ti.nb + P.HL + P.HR;
            const double u0 = (P.t0 - ti.t0h) / P.dt;
            int64_t w_lo;
            int wlen;
            strain_window(P, T, k_lo, ny, u0, &w_lo, &wlen);
            stage_strain(P, ti, hwp, hwc, w_lo, wlen);
            __syncthreads();
            for (int j = threadIdx.x; j < ny; j += blockDim.x) {
                int64_t k = k_lo + j;
                double y[6];
                if (k >= 0 && k < ti.N) {
                    project_sample64<T>(P, skc, k, u0, hwp, hwc, w_lo, wlen, y);
                } else {
#pragma unroll
                    for (int l = 0; l < 6; ++l) y[l] = 0.0;
                }
#pragma unroll
                for (int l = 0; l < 6; ++l) ys[l * P.ymax + j] = y[l];
            }
            __syncthreads();
            double dh = 0.0, hh = 0.0;  // likelihood partials of this thread's outputs
            for (int i = threadIdx.x; i < ti.nb; i += blockDim.x) {
                int64_t n = ti.n0 + i;
                double o[3];
                tdi_sample64<T>(P, n, ys, P.ymax, k_lo, ny, o);
                if (ti.out) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) ti.out[c * ti.N + n] = o[c];
                }
                if (like && ti.dat) {
                    const double da = __ldg(ti.dat + n), de = __ldg(ti.dat + ti.N + n), dT = __ldg(ti.dat + 2 * ti.N + n);
                    if (!(isfinite(da) && isfinite(de) && isfinite(dT))) atomicOr(P.err, ERR_NONFINITE);
                    like_terms(P.like, o[0], o[1], o[2], da, de, dT, dh, hh);
                }
            }
            if (like) {
                block_sum2(dh, hh, red);
                if (threadIdx.x == 0) like_store(P, g, ti.dat ? dh : nan_d(), ti.dat ? hh : nan_d());
            }
        }
        __syncthreads();
    }
}

template <int T>
__global__ void __launch_bounds__(256) k_project64(FwdParams P)
{
    extern __shared__ double sm[];
    double *hwp = sm, *hwc = sm + P.wmax;
    __shared__ TileInfo ti;
    __shared__ SkyConst skc;
    const int64_t total = P.total_tiles >= 0 ? P.total_tiles : P.src.tile_off[P.src.S];
    for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
        if (threadIdx.x == 0) {
            ti = tile_info(P, g, 6);
            skc = make_sky(ti.sky);
            if (!ti.ok) atomicOr(P.err, ERR_OFFSETS);
        }
        __syncthreads();
        if (ti.ok && ti.nb > 0) {
            const int ny = (int)ti.nb;
            const double u0 = (P.t0 - ti.t0h) / P.dt;
            int64_t w_lo;
            int wlen;
            strain_window(P, T, ti.n0, ny, u0, &w_lo, &wlen);
            stage_strain(P, ti, hwp, hwc, w_lo, wlen);
            __syncthreads();
            for (int j = threadIdx.x; j < ny; j += blockDim.x) {
                int64_t k = ti.n0 + j;
                double y[6];
                project_sample64<T>(P, skc, k, u0, hwp, hwc, w_lo, wlen, y);
#pragma unroll
                for (int l = 0; l < 6; ++l) ti.out[l * ti.N + k] = y[l];
            }
        }
        __syncthreads();
    }
}

template <int T>
__global__ void __launch_bounds__(256) k_tdi64(FwdParams P)
{
    extern __shared__ double sm[];
    double *ys = sm;
    __shared__ TileInfo ti;
    const int64_t total = P.total_tiles >= 0 ? P.total_tiles : P.src.tile_off[P.src.S];
    for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
        if (threadIdx.x == 0) {
            ti = tile_info(P, g, 3);
            if (!ti.ok) atomicOr(P.err, ERR_OFFSETS);
        }
        __syncthreads();
        if (ti.ok && ti.nb > 0) {
            const int64_t k_lo = ti.n0 - P.HL;
            const int ny = (int)ti.nb + P.HL + P.HR;
            for (int l = 0; l < 6; ++l) stage(ys + l * P.ymax, ti.yin + l * ti.N, k_lo, ny, ti.N);
            __syncthreads();
            for (int i = threadIdx.x; i < ti.nb; i += blockDim.x) {
                int64_t n = ti.n0 + i;
                double o[3];
                tdi_sample64<T>(P, n, ys, P.ymax, k_lo, ny, o);
#pragma unroll
                for (int c = 0; c < 3; ++c) ti.out[c * ti.N + n] = o[c];
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- dispatch
template <int T>
static void *kernel_ptr(int kind)
{
    switch (kind) {
        case KIND_PROJECT: return (void *)k_project64<T>;
        case KIND_TDI: return (void *)k_tdi64<T>;
        default: return (void *)k_fused64<T>;
    }
}

#define LR_FOR_ORDERS(X) X(1) X(3) X(5) X(7) X(9) X(11) X(13) X(15) X(17) X(19) X(21) X(23) X(25) X(31) X(41)

static void *kernel_for(int kind, int order)
{
    switch (order) {
#define LR_CASE(p) case p: return kernel_ptr<p + 1>(kind);
        LR_FOR_ORDERS(LR_CASE)
#undef LR_CASE
        default: return nullptr;
    }
}

int smem_fwd64(int kind, int order, const FwdParams &P, size_t *smem)
{
    (void)order;
    size_t w = (size_t)P.wmax, y = (size_t)P.ymax;
    *smem = sizeof(double) * (kind == KIND_PROJECT ? 2 * w : kind == KIND_TDI ? 6 * y : 2 * w + 6 * y);
    return 0;
}

int max_blocks_fwd64(int kind, int order, int threads, size_t smem, int *blocks)
{
    void *k = kernel_for(kind, order);
    if (!k) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, threads, smem);
    return (int)e;
}

int launch_fwd64(int kind, int order, const FwdParams &P, int grid, int threads, size_t smem, void *stream)
{
    void *k = kernel_for(kind, order);
    if (!k) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    void *args[] = {(void *)&P};
    e = cudaLaunchKernel(k, dim3(grid), dim3(threads), args, smem, (cudaStream_t)stream);
    return (int)e;
}

bool order_compiled(int order) { return kernel_for(KIND_FUSED, order) != nullptr; }

}  // namespace lr
