// Instantiations of the persistent GADI kernel for the K_2D5 class with the
// SM-resident H-solve (p of CG on H kept in shared memory).
#include "gadi_inst.h"
#include "gadi_solver.cuh"

namespace gadi {
const void *kernel_2d5_res(int prec, int dd)
{
    if (dd) return kernel_2d5_res_dd(prec);
    switch (prec) {
    case P_FP32:
        return (const void *)gadi_stencil_kernel<K_2D5, P_FP32, 4, 2, 1>;
    case P_BF16:
        return (const void *)gadi_stencil_kernel<K_2D5, P_BF16, 8, 2, 1>;
    }
    return nullptr;
}
} // namespace gadi
