// Mixed-precision forward kernels of orders 9, 11, 13, 15.
#include "lr_fwdmx.cuh"

namespace lr {

template <int T>
static void *kernel_ptr_mx(int kind)
{
    switch (kind) {
        case KIND_PROJECT: return (void *)k_mixed<T, KIND_PROJECT>;
        case KIND_TDI: return (void *)k_mixed<T, KIND_TDI>;
        case KIND_LIKE: return (void *)k_mixed<T, KIND_LIKE>;
        default: return (void *)k_mixed<T, KIND_FUSED>;
    }
}

void *kernel_for_mx_p09(int kind, int order)
{
    switch (order) {
        case 9: return kernel_ptr_mx<10>(kind);
        case 11: return kernel_ptr_mx<12>(kind);
        case 13: return kernel_ptr_mx<14>(kind);
        case 15: return kernel_ptr_mx<16>(kind);
        default: return nullptr;
    }
}

}  // namespace lr
