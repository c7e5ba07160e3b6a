// Mixed-precision forward kernels: launch interface.  The kernel instances of each order live
// in lr_fwdmx_pNN.cu (a few orders per file, so that they compile in parallel).
#include "lr_fwdmx.cuh"

namespace lr {

void *kernel_for_mx_p01(int kind, int order);
void *kernel_for_mx_p09(int kind, int order);
void *kernel_for_mx_p17(int kind, int order);
void *kernel_for_mx_p25(int kind, int order);
void *kernel_for_mx_p31(int kind, int order);
void *kernel_for_mx_p41(int kind, int order);

static void *kernel_for_mx(int kind, int order)
{
    switch (order) {
        case 1:
        case 3:
        case 5:
        case 7:
            return kernel_for_mx_p01(kind, order);
        case 9:
        case 11:
        case 13:
        case 15:
            return kernel_for_mx_p09(kind, order);
        case 17:
        case 19:
        case 21:
        case 23:
            return kernel_for_mx_p17(kind, order);
        case 25:
            return kernel_for_mx_p25(kind, order);
        case 31:
            return kernel_for_mx_p31(kind, order);
        case 41:
            return kernel_for_mx_p41(kind, order);
        default: return nullptr;
    }
}

int smem_fwdmx(int kind, int order, const FwdParams &P, size_t *smem)
{
    (void)kind;
    (void)P;
    *smem = (size_t)mx_smem_floats(order + 1) * sizeof(float);
    return 0;
}

int max_blocks_fwdmx(int kind, int order, int threads, size_t smem, int *blocks)
{
    void *k = kernel_for_mx(kind, order);
    if (!k) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, threads, smem);
}

int launch_fwdmx(int kind, int order, const FwdParams &P, int grid, int threads, size_t smem, void *stream)
{
    void *k = kernel_for_mx(kind, order);
    if (!k) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    void *args[] = {(void *)&P};
    return (int)cudaLaunchKernel(k, dim3(grid), dim3(threads), args, smem, (cudaStream_t)stream);
}

bool order_compiled_mx(int order) { return kernel_for_mx(KIND_FUSED, order) != nullptr; }

}  // namespace lr
