// Mixed-precision forward kernels of orders 1, 3, 5, 7.
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

void *kernel_for_mx_p01(int kind, int order)
{
    switch (order) {
        case 1: return kernel_ptr_mx<2>(kind);
        case 3: return kernel_ptr_mx<4>(kind);
        case 5: return kernel_ptr_mx<6>(kind);
        case 7: return kernel_ptr_mx<8>(kind);
        default: return nullptr;
    }
}

}  // namespace lr
