// Batched persistent solve: the lookup of the kernel instantiations (the
// kernel itself is in gadi_batched.cuh).
#include "gadi.h"
#include "gadi_batched.cuh"
#include "gadi_multi.cuh"
#include "gadi_inst.h"

namespace gadi {

const void *kernel_batched4_2d5(size_t *smem)
{
    *smem = 0;
    return (const void *)gadi_batched4_kernel;
}

const void *kernel_batched_2d5_res(int prec)
{
    switch (prec) {
    case P_FP32:
        return (const void *)gadi_batched_kernel<K_2D5, P_FP32, 4, 2, false, 1>;
    case P_BF16:
        return (const void *)gadi_batched_kernel<K_2D5, P_BF16, 8, 2, false, 1>;
    }
    return nullptr;
}

const void *kernel_batched_2d5(int prec, int vec, size_t *smem, int dd)
{
    if (dd) return kernel_batched_2d5_dd(prec, vec, smem);
    switch (prec) {
    case P_FP64:
        *smem = vec ? StencilImpl<K_2D5, P_FP64, 2, 2>::DSMEM : StencilImpl<K_2D5, P_FP64, 1, 1>::DSMEM;
        return vec ? (const void *)gadi_batched_kernel<K_2D5, P_FP64, 2, 2>
                   : (const void *)gadi_batched_kernel<K_2D5, P_FP64, 1, 1>;
    case P_FP32:
        *smem = vec ? StencilImpl<K_2D5, P_FP32, 4, 2>::DSMEM : StencilImpl<K_2D5, P_FP32, 1, 1>::DSMEM;
        return vec ? (const void *)gadi_batched_kernel<K_2D5, P_FP32, 4, 2>
                   : (const void *)gadi_batched_kernel<K_2D5, P_FP32, 1, 1>;
    case P_BF16:
        *smem = vec ? StencilImpl<K_2D5, P_BF16, 8, 2>::DSMEM : StencilImpl<K_2D5, P_BF16, 1, 1>::DSMEM;
        return vec ? (const void *)gadi_batched_kernel<K_2D5, P_BF16, 8, 2>
                   : (const void *)gadi_batched_kernel<K_2D5, P_BF16, 1, 1>;
    }
    *smem = 0;
    return nullptr;
}

} // namespace gadi
