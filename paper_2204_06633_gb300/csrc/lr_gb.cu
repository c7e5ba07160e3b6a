// Galactic-binary polarisations on the device as arrays (the same generator the fused kernels
// use when the strain is generated on chip; Sec. "Template generation").
#include <cuda_runtime.h>

#include <cmath>

#include "lr_gb.cuh"

namespace lr {
namespace {

__global__ void k_gb_polarisations(GbConst g, double t0, double dt, int64_t n, double *__restrict__ hp,
                                   double *__restrict__ hc)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        gb_strain(g, t0, dt, i, hp[i], hc[i]);
}

}  // namespace
}  // namespace lr

extern "C" LR_API int lr_gb_polarisations(const lr_gb *gb, double t0, double dt, int64_t n, double *hp, double *hc,
                                          void *stream)
{
    if (!gb || !hp || !hc || n < 0) return LR_ERR_INVALID_ARG;
    if (!std::isfinite(gb->A) || !std::isfinite(gb->f0) || !std::isfinite(gb->fdot) || !std::isfinite(gb->fddot) ||
        !std::isfinite(gb->phi0) || !std::isfinite(gb->iota) || !std::isfinite(t0) || !std::isfinite(dt))
        return LR_ERR_NONFINITE;
    if (n > ((int64_t)1 << 50)) return LR_ERR_RANGE;
    if (n == 0) return LR_OK;
    const int64_t blocks = (n + 255) / 256;
    lr::k_gb_polarisations<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, (cudaStream_t)stream>>>(
        lr::make_gb(*gb), t0, dt, n, hp, hc);
    return cudaGetLastError() == cudaSuccess ? LR_OK : LR_ERR_CUDA;
}
