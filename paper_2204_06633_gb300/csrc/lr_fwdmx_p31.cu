// Mixed-precision forward kernels of order 31.
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

void *kernel_for_mx_p31(int kind, int order)
{
    switch (order) {
        case 31: return kernel_ptr_mx<32>(kind);
        default: return nullptr;
    }
}

}  // namespace lr
