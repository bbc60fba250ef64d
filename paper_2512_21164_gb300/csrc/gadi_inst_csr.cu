// Instantiations of the persistent GADI kernel for general CSR matrices.
#include "gadi_inst.h"
#include "gadi_solver.cuh"

namespace gadi {
const void *kernel_csr(int prec, int dd)
{
    switch (prec) {
    case P_FP64: return dd ? (const void *)gadi_csr_kernel<P_FP64, true> : (const void *)gadi_csr_kernel<P_FP64>;
    case P_FP32: return dd ? (const void *)gadi_csr_kernel<P_FP32, true> : (const void *)gadi_csr_kernel<P_FP32>;
    case P_BF16: return dd ? (const void *)gadi_csr_kernel<P_BF16, true> : (const void *)gadi_csr_kernel<P_BF16>;
    }
    return nullptr;
}
} // namespace gadi
