// Instantiations of the persistent GADI kernel for the C2D5 class with the
// residual in double-FP64 (u_r ~ u^2).
#include "gadi_inst.h"
#include "gadi_solver.cuh"

namespace gadi {
const void *kernel_c2d5_dd(int prec, int vec)
{
    switch (prec) {
    case P_FP64:
        return (const void *)gadi_stencil_kernel<K_C2D5, P_FP64, 2, 2, 0, true>;
    case P_FP32:
        return vec ? (const void *)gadi_stencil_kernel<K_C2D5, P_FP32, 4, 2, 0, true>
                   : (const void *)gadi_stencil_kernel<K_C2D5, P_FP32, 2, 2, 0, true>;
    case P_BF16:
        return vec ? (const void *)gadi_stencil_kernel<K_C2D5, P_BF16, 8, 2, 0, true>
                   : (const void *)gadi_stencil_kernel<K_C2D5, P_BF16, 2, 2, 0, true>;
    }
    return nullptr;
}
} // namespace gadi
