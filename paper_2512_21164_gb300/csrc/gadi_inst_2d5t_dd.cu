// Instantiations of the persistent GADI kernel for the K_2D5 class with the
// tensor-memory H-solve and the residual in double-FP64 (u_r ~ u^2).
#include "gadi_inst.h"
#include "gadi_solver.cuh"

namespace gadi {
const void *kernel_2d5_tm_dd(int prec)
{
    switch (prec) {
    case P_FP32:
        return (const void *)gadi_stencil_kernel<K_2D5, P_FP32, 4, 2, 2, true>;
    case P_BF16:
        return (const void *)gadi_stencil_kernel<K_2D5, P_BF16, 8, 2, 2, true>;
    }
    return nullptr;
}
} // namespace gadi
