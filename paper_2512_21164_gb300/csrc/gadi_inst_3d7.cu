// Instantiations of the persistent GADI kernel for the K_3D7 class.
#include "gadi_inst.h"
#include "gadi_solver.cuh"

namespace gadi {
const void *kernel_3d7(int prec, int vec, int dd)
{
    if (dd) return kernel_3d7_dd(prec, vec);
    switch (prec) {
    case P_FP64:
        return vec ? (const void *)gadi_stencil_kernel<K_3D7, P_FP64, 2, 2>
                   : (const void *)gadi_stencil_kernel<K_3D7, P_FP64, 1, 1>;
    case P_FP32:
        return vec ? (const void *)gadi_stencil_kernel<K_3D7, P_FP32, 4, 2>
                   : (const void *)gadi_stencil_kernel<K_3D7, P_FP32, 1, 1>;
    case P_BF16:
        return vec ? (const void *)gadi_stencil_kernel<K_3D7, P_BF16, 8, 2>
                   : (const void *)gadi_stencil_kernel<K_3D7, P_BF16, 1, 1>;
    }
    return nullptr;
}
size_t kernel_3d7_smem(int prec, int vec)
{
    switch (prec) {
    case P_FP64:
        return vec ? StencilImpl<K_3D7, P_FP64, 2, 2>::DSMEM : StencilImpl<K_3D7, P_FP64, 1, 1>::DSMEM;
    case P_FP32:
        return vec ? StencilImpl<K_3D7, P_FP32, 4, 2>::DSMEM : StencilImpl<K_3D7, P_FP32, 1, 1>::DSMEM;
    case P_BF16:
        return vec ? StencilImpl<K_3D7, P_BF16, 8, 2>::DSMEM : StencilImpl<K_3D7, P_BF16, 1, 1>::DSMEM;
    }
    return 0;
}
} // namespace gadi
