// Instantiations of the persistent GADI kernel for the complex 2D class
// (interleaved re/im: two elements per grid point).
#include "gadi_inst.h"
#include "gadi_solver.cuh"

namespace gadi {
const void *kernel_c2d5(int prec, int vec, int dd)
{
    if (dd) return kernel_c2d5_dd(prec, vec);
    switch (prec) {
    case P_FP64:
        return (const void *)gadi_stencil_kernel<K_C2D5, P_FP64, 2, 2>;
    case P_FP32:
        return vec ? (const void *)gadi_stencil_kernel<K_C2D5, P_FP32, 4, 2>
                   : (const void *)gadi_stencil_kernel<K_C2D5, P_FP32, 2, 2>;
    case P_BF16:
        return vec ? (const void *)gadi_stencil_kernel<K_C2D5, P_BF16, 8, 2>
                   : (const void *)gadi_stencil_kernel<K_C2D5, P_BF16, 2, 2>;
    }
    return nullptr;
}
size_t kernel_c2d5_smem(int prec, int vec)
{
    switch (prec) {
    case P_FP64:
        return StencilImpl<K_C2D5, P_FP64, 2, 2>::DSMEM;
    case P_FP32:
        return vec ? StencilImpl<K_C2D5, P_FP32, 4, 2>::DSMEM : StencilImpl<K_C2D5, P_FP32, 2, 2>::DSMEM;
    case P_BF16:
        return vec ? StencilImpl<K_C2D5, P_BF16, 8, 2>::DSMEM : StencilImpl<K_C2D5, P_BF16, 2, 2>::DSMEM;
    }
    return 0;
}
} // namespace gadi
