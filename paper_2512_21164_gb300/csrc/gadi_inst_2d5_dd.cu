// Instantiations of the persistent GADI kernel for the 2D5 class with the
// residual in double-FP64 (u_r ~ u^2).
#include "gadi_inst.h"
#include "gadi_solver.cuh"

namespace gadi {
const void *kernel_2d5_dd(int prec, int vec)
{
    switch (prec) {
    case P_FP64:
        return vec ? (const void *)gadi_stencil_kernel<K_2D5, P_FP64, 2, 2, 0, true>
                   : (const void *)gadi_stencil_kernel<K_2D5, P_FP64, 1, 1, 0, true>;
    case P_FP32:
        return vec ? (const void *)gadi_stencil_kernel<K_2D5, P_FP32, 4, 2, 0, true>
                   : (const void *)gadi_stencil_kernel<K_2D5, P_FP32, 1, 1, 0, true>;
    case P_BF16:
        return vec ? (const void *)gadi_stencil_kernel<K_2D5, P_BF16, 8, 2, 0, true>
                   : (const void *)gadi_stencil_kernel<K_2D5, P_BF16, 1, 1, 0, true>;
    }
    return nullptr;
}
const void *kernel_2d5_res_dd(int prec)
{
    switch (prec) {
    case P_FP32:
        return (const void *)gadi_stencil_kernel<K_2D5, P_FP32, 4, 2, 1, true>;
    case P_BF16:
        return (const void *)gadi_stencil_kernel<K_2D5, P_BF16, 8, 2, 1, true>;
    }
    return nullptr;
}
} // namespace gadi
