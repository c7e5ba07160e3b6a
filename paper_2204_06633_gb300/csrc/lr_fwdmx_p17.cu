// Mixed-precision forward kernels of orders 17, 19, 21, 23.
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

void *kernel_for_mx_p17(int kind, int order)
{
    switch (order) {
        case 17: return kernel_ptr_mx<18>(kind);
        case 19: return kernel_ptr_mx<20>(kind);
        case 21: return kernel_ptr_mx<22>(kind);
        case 23: return kernel_ptr_mx<24>(kind);
        default: return nullptr;
    }
}

}  // namespace lr
