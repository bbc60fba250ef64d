// gadi_solve_h_2d_noalloc: the H-solve (CG on alpha I + M for the 2D 5-point
// class) for callers that cannot allocate device memory -- for example code
// running where cudaMalloc is unavailable or forbidden (inside a pre-sized
// memory pool, a plug-in host that owns every allocation, or a process that
// must not grow its device footprint after start-up).  Its work vectors and
// control words live in one file-scope device array instead of memory from
// cudaMalloc; the caller still passes the right-hand side and the result.
#include "gadi.h"
#include "gadi_inst.h"
#include "gadi_params.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

using namespace gadi;

namespace {

constexpr long long kNoAllocMaxElems = 262144; // e.g. a 512 x 512 grid
constexpr int kNoAllocMaxBlocks = 2048;
constexpr int kThreadsNA = GADI_THREADS; // block size of the persistent kernel
constexpr size_t kSlab = (size_t)kNoAllocMaxElems * 8; // one vector at FP64, the widest u_s
constexpr size_t kPartBytes = sizeof(double) * 4 * kNoAllocMaxBlocks;
constexpr size_t kCtlBytes = 256, kHistBytes = 256, kBarBytes = 256, kAbortBytes = 256;
constexpr size_t kScratchBytes = 5 * kSlab + kPartBytes + kCtlBytes + kHistBytes + kBarBytes + kAbortBytes;

// The scratch itself: every GPU that loads the library holds it (about
// 10.6 MB) until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct ScratchSlot {
    unsigned long long ctx_id; // context the address belongs to (0: none yet)
    void *addr;
};
ScratchSlot g_slot[kMaxDevices] = {};

// Driver entry points for the identity of the current context, resolved once
// through the runtime (no link against the driver library).  Each context
// gets a process-unique id, so a context rebuilt after cudaDeviceReset (in
// which the module, and with it the array, may sit elsewhere) never matches
// an old entry.
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_ctx_fns_tried = false;

// id of the current context, 0 if it cannot be told (then the address is
// looked up again on every call)
unsigned long long current_context_id()
{
    if (!g_ctx_fns_tried) {
        g_ctx_fns_tried = true;
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            g_ctx_current = (CtxGetCurrentFn)f1;
            g_ctx_id = (CtxGetIdFn)f2;
        }
        cudaGetLastError();
    }
    if (!g_ctx_current || !g_ctx_id) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&ctx) != 0 || !ctx || g_ctx_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of the scratch on the current device.  In host code the
// symbol names a host-side stand-in, never the device memory, so the address
// comes from cudaGetSymbolAddress: once per device (and context), with that
// device current.
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    unsigned long long id = current_context_id();
    if (id != 0 && g_slot[dev].ctx_id == id && g_slot[dev].addr) {
        *out = g_slot[dev].addr;
        return cudaSuccess;
    }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch); // creates the context if there is none yet
    if (e != cudaSuccess) return e;
    if (id == 0) id = current_context_id();
    g_slot[dev].ctx_id = id;
    g_slot[dev].addr = p;
    *out = p;
    return cudaSuccess;
}

// u_s rounding of the H diagonal (same definition as the handle-based path:
// round to nearest even; BF16 via round-to-odd at binary32 first)
double na_round_us(int prec, double v)
{
    if (prec == P_FP32) return (double)(float)v;
    if (prec != P_BF16) return v;
    float f = (float)v;
    if ((double)f != v && std::isfinite(v)) {
        if (std::fabs((double)f) > std::fabs(v)) f = std::nextafter(f, 0.0f);
        uint32_t u;
        std::memcpy(&u, &f, 4);
        u |= 1u;
        std::memcpy(&f, &u, 4);
    }
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return v;
    u += 0x7fffu + ((u >> 16) & 1u);
    u &= 0xffff0000u;
    std::memcpy(&f, &u, 4);
    return (double)f;
}

gadi_status na_fail(cudaError_t e, const char *what)
{
    char buf[200];
    std::snprintf(buf, sizeof buf, "gadi_solve_h_2d_noalloc: %s: %s", what, cudaGetErrorString(e));
    record_error(buf);
    return GADI_ERR_CUDA;
}

} // namespace

extern "C" gadi_status gadi_solve_h_2d_noalloc(int nx, int ny, double alpha, gadi_prec u_low, const void *rs,
                                               void *z, double tol, int maxit, int stag, int *its, void *stream)
{
    if (nx <= 0 || ny <= 0 || !rs || !z || !(alpha > 0) || !std::isfinite(alpha) || !(tol >= 0) || maxit < 0 ||
        stag < 0)
        return GADI_ERR_INVALID;
    if (u_low != GADI_FP64 && u_low != GADI_FP32 && u_low != GADI_BF16) return GADI_ERR_INVALID;
    const long long n = (long long)nx * ny;
    if (n > kNoAllocMaxElems) {
        char buf[200];
        std::snprintf(buf, sizeof buf,
                      "gadi_solve_h_2d_noalloc: %lld grid points exceed the static scratch maximum of %lld",
                      n, kNoAllocMaxElems);
        record_error(buf);
        return GADI_ERR_INVALID;
    }
    const int prec = (int)u_low;
    const size_t eb = prec == P_FP64 ? 8 : (prec == P_FP32 ? 4 : 2);
    cudaStream_t st = (cudaStream_t)stream;

    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return na_fail(e, "cudaGetSymbolAddress");
    char *b = (char *)base;
    void *slab[5];
    for (int i = 0; i < 5; i++) slab[i] = b + (size_t)i * kSlab;
    char *tail = b + 5 * kSlab;
    double *part = (double *)tail;
    Ctl *ctl = (Ctl *)(tail + kPartBytes);
    double *hist = (double *)(tail + kPartBytes + kCtlBytes);
    unsigned long long *bar = (unsigned long long *)(tail + kPartBytes + kCtlBytes + kHistBytes);
    int *abort_flag = (int *)(tail + kPartBytes + kCtlBytes + kHistBytes + kBarBytes);

    int dev = 0, nsm = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return na_fail(e, "cudaGetDevice");
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return na_fail(e, "cudaDeviceGetAttribute");
    const int vec_elems = prec == P_FP64 ? 2 : (prec == P_FP32 ? 4 : 8);
    const bool vec = (nx % vec_elems) == 0 && ((uintptr_t)z & 15u) == 0;
    const void *kern = kernel_2d5(prec, vec ? 1 : 0);
    const size_t smem = kernel_2d5_smem(prec, vec ? 1 : 0);
    if (smem && (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
                    cudaSuccess)
        return na_fail(e, "cudaFuncSetAttribute");
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreadsNA, smem)) != cudaSuccess)
        return na_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    int blocks = per_sm * nsm;
    if (blocks > kNoAllocMaxBlocks) blocks = kNoAllocMaxBlocks;
    if (blocks <= 0) return GADI_ERR_CUDA;

    Params P;
    std::memset(&P, 0, sizeof P);
    P.kind = K_2D5;
    P.prec = prec;
    P.mode = MODE_SOLVE_H;
    P.nx = nx;
    P.ny = ny;
    P.nz = 1;
    P.npts = P.nelem = n;
    P.co.h_d = na_round_us(prec, alpha + 4.0); // H = alpha I + M, M: centre 4, neighbours -1
    for (int k = 0; k < 4; k++) P.co.h_c[k] = -1.0;
    P.r = slab[0];
    P.p0 = slab[1];
    P.p1 = slab[2];
    P.u = slab[3];
    P.y = slab[4];
    P.z = z;
    P.tol_h = tol;
    P.maxit_inner = maxit;
    P.inner_stag = stag;
    P.maxit = 1;
    P.part = part;
    P.hist = hist;
    P.ctl = ctl;
    P.bar = bar;
    P.abort_flag = abort_flag;

    // the scratch keeps the previous call's contents: clear what must start at zero
    if ((e = cudaMemsetAsync(bar, 0, kBarBytes, st)) != cudaSuccess) return na_fail(e, "cudaMemsetAsync");
    if ((e = cudaMemsetAsync(abort_flag, 0, kAbortBytes, st)) != cudaSuccess) return na_fail(e, "cudaMemsetAsync");
    if ((e = cudaMemsetAsync(ctl, 0, kCtlBytes, st)) != cudaSuccess) return na_fail(e, "cudaMemsetAsync");
    if ((e = cudaMemcpyAsync(slab[0], rs, eb * (size_t)n, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return na_fail(e, "cudaMemcpyAsync");
    void *args[] = {&P};
    fill_coef_sets(P);
    if ((e = cudaLaunchCooperativeKernel(kern, dim3(blocks), dim3(kThreadsNA), args, smem, st)) != cudaSuccess)
        return na_fail(e, "cudaLaunchCooperativeKernel");
    Ctl hc;
    int hab = 0;
    if ((e = cudaMemcpyAsync(&hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return na_fail(e, "cudaMemcpyAsync");
    if ((e = cudaMemcpyAsync(&hab, abort_flag, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return na_fail(e, "cudaMemcpyAsync");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return na_fail(e, "cudaStreamSynchronize");
    if (hab) return GADI_ERR_TIMEOUT;
    if (its) *its = (int)hc.inner_h;
    return GADI_OK;
}
