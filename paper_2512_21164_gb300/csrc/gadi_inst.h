// Kernel lookup across the per-class translation units.
#pragma once
#include <cstddef>
namespace gadi {
// vec = 1 selects the 16-byte vector path (requires the row length in
// elements to be a multiple of the elements per 16 bytes), 0 the narrow path.
// dd = 1 selects the instantiation whose residual is in double-FP64.
const void *kernel_2d5(int prec, int vec, int dd = 0);
// the 2D kernel with the SM-resident H-solve (FP32/BF16, 16-byte path; else null)
const void *kernel_2d5_res(int prec, int dd = 0);
// the same with z and r of the H-solve in tensor memory
const void *kernel_2d5_tm(int prec, int dd = 0);
const void *kernel_3d7(int prec, int vec, int dd = 0);
const void *kernel_c2d5(int prec, int vec, int dd = 0);
const void *kernel_csr(int prec, int dd = 0);
const void *kernel_2d5_dd(int prec, int vec);
const void *kernel_2d5_res_dd(int prec);
const void *kernel_2d5_tm_dd(int prec);
const void *kernel_3d7_dd(int prec, int vec);
const void *kernel_c2d5_dd(int prec, int vec);
// dynamic shared memory (bytes) the selected stencil kernel needs at launch
size_t kernel_2d5_smem(int prec, int vec);
size_t kernel_3d7_smem(int prec, int vec);
size_t kernel_c2d5_smem(int prec, int vec);
// the batched persistent kernel for the 2D 5-point class
const void *kernel_batched_2d5(int prec, int vec, size_t *smem, int dd = 0);
const void *kernel_batched_2d5_dd(int prec, int vec, size_t *smem);
// the batched kernel with units of four interleaved right-hand sides (FP32)
const void *kernel_batched4_2d5(size_t *smem);
// the batched kernel whose units take the SM-resident H-solve (FP32 / BF16,
// 16-byte rows; dynamic shared memory set by the caller)
const void *kernel_batched_2d5_res(int prec);
// record a message for gadi_last_error() on this thread
void record_error(const char *msg);
} // namespace gadi
