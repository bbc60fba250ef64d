// Batched persistent solve with the residual in double-FP64 (u_r ~ u^2).
#include "gadi.h"
#include "gadi_batched.cuh"
#include "gadi_inst.h"

namespace gadi {

const void *kernel_batched_2d5_dd(int prec, int vec, size_t *smem)
{
    switch (prec) {
    case P_FP64:
        *smem = vec ? StencilImpl<K_2D5, P_FP64, 2, 2>::DSMEM : StencilImpl<K_2D5, P_FP64, 1, 1>::DSMEM;
        return vec ? (const void *)gadi_batched_kernel<K_2D5, P_FP64, 2, 2, true>
                   : (const void *)gadi_batched_kernel<K_2D5, P_FP64, 1, 1, true>;
    case P_FP32:
        *smem = vec ? StencilImpl<K_2D5, P_FP32, 4, 2>::DSMEM : StencilImpl<K_2D5, P_FP32, 1, 1>::DSMEM;
        return vec ? (const void *)gadi_batched_kernel<K_2D5, P_FP32, 4, 2, true>
                   : (const void *)gadi_batched_kernel<K_2D5, P_FP32, 1, 1, true>;
    case P_BF16:
        *smem = vec ? StencilImpl<K_2D5, P_BF16, 8, 2>::DSMEM : StencilImpl<K_2D5, P_BF16, 1, 1>::DSMEM;
        return vec ? (const void *)gadi_batched_kernel<K_2D5, P_BF16, 8, 2, true>
                   : (const void *)gadi_batched_kernel<K_2D5, P_BF16, 1, 1, true>;
    }
    *smem = 0;
    return nullptr;
}

} // namespace gadi
