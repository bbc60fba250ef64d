// Host side of the C ABI declared in include/gadi.h: handle management,
// argument validation, the operator coefficients of the HSS splitting
// (rounded to u_s), workspace, host/device pointer staging and the
// cooperative launches of the persistent kernel.
#include "gadi.h"
#include "gadi_inst.h"
#include "gadi_params.h"
#include "gadi_common.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

using namespace gadi;

namespace {

constexpr int kThreadsHost = GADI_THREADS; // = gadi::kThreads

// --------------------------------------------------------------------------
// host-side rounding of FP64 scalars to the storage precision u_s
// --------------------------------------------------------------------------
// BF16: first round to odd at binary32 (take the nearest float, step it one
// unit toward zero if it rounded away, and mark any inexactness in its last
// bit), then round to nearest even at 8 significant bits on the bit pattern.
uint16_t host_f32_to_bf16(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float host_bf16_to_f32(uint16_t b)
{
    uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}
float host_round_odd_f32(double d)
{
    if (std::isnan(d) || std::isinf(d)) return (float)d;
    float f = (float)d;
    if ((double)f == d) return f;
    if (std::fabs((double)f) > std::fabs(d)) f = std::nextafter(f, 0.0f);
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u |= 1u;
    std::memcpy(&f, &u, 4);
    return f;
}
double round_us(int prec, double v)
{
    if (prec == P_FP32) return (double)(float)v;
    if (prec == P_BF16) return (double)host_bf16_to_f32(host_f32_to_bf16(host_round_odd_f32(v)));
    return v;
}
double round_compute(int prec, double v) { return prec == P_FP64 ? v : (double)(float)v; }
size_t elem_bytes(int prec) { return prec == P_FP64 ? 8 : (prec == P_FP32 ? 4 : 2); }
size_t compute_bytes(int prec) { return prec == P_FP64 ? 8 : 4; }

struct Stencil {
    double d, c[6], e;
};

} // namespace

struct gadi_handle {
    int kind = 0, nx = 0, ny = 0, nz = 0;
    long long npts = 0, nelem = 0;
    double h = 0, beta[3] = {0, 0, 0}, kappa = 0, sigma = 0;
    Stencil A{}, M{}, N{};
    int device = 0, nsm = 0;
    // CSR
    int nnz = 0, nnzm = 0;
    int *d_rowptr = nullptr, *d_col = nullptr, *d_mrowptr = nullptr, *d_mcol = nullptr;
    double *d_aval = nullptr, *d_mval = nullptr, *d_nval = nullptr, *d_atval = nullptr;
    std::vector<int> h_mrowptr, h_mcol;
    std::vector<double> h_mval, h_nval;
    void *d_opval = nullptr; // H, S, S^T values in u_s (3 * nnzm elements)
    int op_prec = -1;
    double op_alpha = NAN;
    // workspace
    void *d_ws = nullptr;
    size_t ws_bytes = 0;
    double *d_part = nullptr, *d_hist = nullptr;
    int part_cap = 0, hist_cap = 0;
    Ctl *d_ctl = nullptr, *h_ctl = nullptr;
    unsigned long long *d_bar = nullptr;
    int *d_abort = nullptr, *d_flag = nullptr, *h_flag = nullptr;
    double *d_stage = nullptr; // 2 * nelem doubles for host b / x
    double *d_pw = nullptr;    // power-iteration vectors (3 * nelem)
    double *d_sig = nullptr;   // complex class: per-point T (npts), or null
    double *d_acc = nullptr;   // two doubles: device sums for the backward error
    double anorm = -1.0;       // ||A||_2 estimate kept for the backward error
    int anorm_iters = 0;       // power-iteration steps it was taken with
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

thread_local char g_last_error[256] = "";

gadi_status cuda_err(cudaError_t e, const char *what, int line)
{
    std::snprintf(g_last_error, sizeof g_last_error, "%s (line %d): %s", what, line, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? GADI_ERR_OOM : GADI_ERR_CUDA;
}
#define CK(call)                                                                                             \
    do {                                                                                                     \
        cudaError_t e_ = (call);                                                                             \
        if (e_ != cudaSuccess) return cuda_err(e_, #call, __LINE__);                                          \
    } while (0)

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void stencil_coefs(gadi_handle *h)
{
    const double cx = h->beta[0] * h->h / 2.0, cy = h->beta[1] * h->h / 2.0, cz = h->beta[2] * h->h / 2.0;
    Stencil M{}, N{};
    if (h->kind == GADI_STENCIL_2D5) {
        M.d = 4.0 + h->kappa;
        for (int k = 0; k < 4; k++) M.c[k] = -1.0;
        N.c[0] = -cx; N.c[1] = cx; N.c[2] = -cy; N.c[3] = cy;
    } else if (h->kind == GADI_STENCIL_3D7) {
        M.d = 6.0 + h->kappa;
        for (int k = 0; k < 6; k++) M.c[k] = -1.0;
        N.c[0] = -cx; N.c[1] = cx; N.c[2] = -cy; N.c[3] = cy; N.c[4] = -cz; N.c[5] = cz;
    } else {
        M.d = 4.0 + h->kappa;
        for (int k = 0; k < 4; k++) M.c[k] = -1.0;
        N.e = h->sigma;
    }
    Stencil A{};
    A.d = M.d + N.d;
    for (int k = 0; k < 6; k++) A.c[k] = M.c[k] + N.c[k];
    A.e = M.e + N.e;
    h->A = A;
    h->M = M;
    h->N = N;
}

gadi_status ensure_ctl(gadi_handle *h, int blocks, int maxit)
{
    if (!h->d_ctl) {
        CK(cudaMalloc(&h->d_ctl, sizeof(Ctl)));
        CK(cudaMallocHost(&h->h_ctl, sizeof(Ctl)));
        CK(cudaMalloc(&h->d_bar, 64));
        CK(cudaMalloc(&h->d_abort, 64));
        CK(cudaMalloc(&h->d_flag, 64));
        CK(cudaMallocHost(&h->h_flag, 64));
        CK(cudaEventCreate(&h->ev0));
        CK(cudaEventCreate(&h->ev1));
    }
    if (blocks > h->part_cap) {
        if (h->d_part) cudaFree(h->d_part);
        h->d_part = nullptr;
        CK(cudaMalloc(&h->d_part, sizeof(double) * 4 * (size_t)blocks));
        h->part_cap = blocks;
    }
    if (maxit + 2 > h->hist_cap) {
        if (h->d_hist) cudaFree(h->d_hist);
        h->d_hist = nullptr;
        CK(cudaMalloc(&h->d_hist, sizeof(double) * (size_t)(maxit + 2)));
        h->hist_cap = maxit + 2;
    }
    return GADI_OK;
}

// workspace layout: x1 (FP64), then r, z, p0, p1, y, u in u_s, then q in the
// compute type (CSR only), each slab aligned to 256 bytes
struct Work {
    double *x1;
    void *r, *z, *p0, *p1, *y, *u, *q;
};
size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

gadi_status ensure_ws(gadi_handle *h, int prec, Work *w)
{
    const size_t m = (size_t)h->nelem;
    const size_t sv = align256(m * elem_bytes(prec)), dv = align256(m * 8), cv = align256(m * compute_bytes(prec));
    const size_t need = dv + 6 * sv + (h->kind == GADI_CSR ? cv : 0);
    if (need > h->ws_bytes) {
        if (h->d_ws) cudaFree(h->d_ws);
        h->d_ws = nullptr;
        h->ws_bytes = 0;
        CK(cudaMalloc(&h->d_ws, need));
        h->ws_bytes = need;
    }
    char *b = (char *)h->d_ws;
    w->x1 = (double *)b;
    b += dv;
    void **slots[6] = {&w->r, &w->z, &w->p0, &w->p1, &w->y, &w->u};
    for (int i = 0; i < 6; i++) {
        *slots[i] = b;
        b += sv;
    }
    w->q = h->kind == GADI_CSR ? (void *)b : nullptr;
    return GADI_OK;
}

// Every mode gets every work buffer; entry points then point the slots that
// carry caller vectors at those.  No kernel path can meet a null work slot.
void set_work(Params &P, const Work &w)
{
    P.x1 = w.x1;
    P.r = w.r;
    P.z = w.z;
    P.p0 = w.p0;
    P.p1 = w.p1;
    P.y = w.y;
    P.u = w.u;
    P.q = w.q;
}

// u_s copies of H = alpha I + M, S = alpha I + N and S^T = alpha I - N on M's
// pattern (CSR only); the shift is added in FP64 before rounding.
gadi_status ensure_csr_ops(gadi_handle *h, int prec, double alpha)
{
    if (h->op_prec == prec && h->op_alpha == alpha) return GADI_OK;
    const int n = (int)h->npts, nnz = h->nnzm;
    std::vector<double> hv(nnz), sv(nnz), tv(nnz);
    for (int i = 0; i < n; i++)
        for (int k = h->h_mrowptr[i]; k < h->h_mrowptr[i + 1]; k++) {
            const double sh = h->h_mcol[k] == i ? alpha : 0.0;
            hv[k] = round_us(prec, h->h_mval[k] + sh);
            sv[k] = round_us(prec, h->h_nval[k] + sh);
            tv[k] = round_us(prec, sh - h->h_nval[k]);
        }
    const size_t eb = elem_bytes(prec);
    std::vector<unsigned char> buf(3 * (size_t)nnz * eb + 16);
    for (int part = 0; part < 3; part++) {
        const std::vector<double> &src = part == 0 ? hv : (part == 1 ? sv : tv);
        unsigned char *dst = buf.data() + (size_t)part * nnz * eb;
        for (int k = 0; k < nnz; k++) {
            if (prec == P_FP64) {
                std::memcpy(dst + 8 * (size_t)k, &src[k], 8);
            } else if (prec == P_FP32) {
                float f = (float)src[k];
                std::memcpy(dst + 4 * (size_t)k, &f, 4);
            } else {
                uint16_t b = host_f32_to_bf16((float)src[k]); // exact: already a BF16 value
                std::memcpy(dst + 2 * (size_t)k, &b, 2);
            }
        }
    }
    if (h->d_opval) cudaFree(h->d_opval);
    h->d_opval = nullptr;
    h->op_prec = -1;
    CK(cudaMalloc(&h->d_opval, buf.size()));
    CK(cudaMemcpy(h->d_opval, buf.data(), buf.size(), cudaMemcpyHostToDevice));
    h->op_prec = prec;
    h->op_alpha = alpha;
    return GADI_OK;
}

bool aligned16(const void *p) { return p == nullptr || ((uintptr_t)p & 15u) == 0; }

// Every vector the kernel reads or writes with 16-byte loads must start on a
// 16-byte boundary; the narrow path needs only the element alignment, except
// for complex FP64 points (16 bytes), which always need 16.
bool params_aligned(const Params &P)
{
    const void *ps[] = {P.b, P.x, P.x1, P.r_out, P.r, P.z, P.p0, P.p1, P.y, P.u, P.ax_in, P.ax_out};
    for (const void *p : ps)
        if (!aligned16(p)) return false;
    return true;
}

// TMEM slots per thread of the tensor-memory H-solve: 512 columns shared by
// the kThreads / 128 warps of a lane quarter, 8 columns (z and r) a slot
constexpr int kTmSlots = 512 / (kThreadsHost / 128) / 8;

// slots the tensor-memory H-solve needs per thread: the column passes times
// the march steps of the block with the most rows (the device's res_map)
long long tm_slots(long long nxw, long long ny, long long blocks)
{
    long long worst = 0;
    for (long long b = 0; b < blocks; ++b) {
        const long long R = (b + 1) * ny / blocks - b * ny / blocks;
        long long need;
        if (nxw >= kThreadsHost) {
            need = ((nxw + kThreadsHost - 1) / kThreadsHost) * R;
        } else {
            const long long np = kThreadsHost / nxw;
            need = (R + np - 1) / np;
        }
        worst = std::max(worst, need);
    }
    return worst;
}

const void *pick_kernel(gadi_handle *h, int prec, bool aligned, size_t *smem, int *vec_out = nullptr, int dd = 0)
{
    *smem = 0;
    if (vec_out) *vec_out = 0;
    if (h->kind == GADI_CSR) return kernel_csr(prec, dd);
    const long long ne = (long long)h->nx * (h->kind == GADI_COMPLEX_2D5 ? 2 : 1);
    const int vec = prec == P_FP64 ? 2 : (prec == P_FP32 ? 4 : 8);
    const int v = aligned && (ne % vec) == 0;
    if (vec_out) *vec_out = v;
    if (h->kind == GADI_STENCIL_2D5) {
        *smem = kernel_2d5_smem(prec, v);
        return kernel_2d5(prec, v, dd);
    }
    if (h->kind == GADI_STENCIL_3D7) {
        *smem = kernel_3d7_smem(prec, v);
        return kernel_3d7(prec, v, dd);
    }
    *smem = kernel_c2d5_smem(prec, v);
    return kernel_c2d5(prec, v, dd);
}

gadi_status launch(gadi_handle *h, int prec, Params &P, int max_blocks, cudaStream_t st, int *blocks_out)
{
    // refuse to launch with a null slot the mode dereferences
    if (P.mode == MODE_SOLVE || P.mode == MODE_SOLVE_H || P.mode == MODE_SOLVE_S) {
        if (!P.r || !P.z || !P.p0 || !P.p1 || !P.y || !P.u || (h->kind == GADI_CSR && !P.q))
            return GADI_ERR_INVALID;
    }
    if ((P.mode == MODE_SOLVE || P.mode == MODE_RESIDUAL) && (!P.b || !P.x || !P.x1 || !P.r))
        return GADI_ERR_INVALID;
    if (P.mode == MODE_APPLY && (!P.ax_in || !P.ax_out)) return GADI_ERR_INVALID;
    const bool al = params_aligned(P);
    if (!al && h->kind == GADI_COMPLEX_2D5) return GADI_ERR_INVALID; // complex vectors: 16-byte aligned
    size_t smem = 0;
    int vec = 0;
    const void *k = pick_kernel(h, prec, al, &smem, &vec, P.ur_dd);
    if (!k) return GADI_ERR_UNSUPPORTED;
    if (smem) CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreadsHost, smem));
    if (per_sm <= 0) return GADI_ERR_CUDA;
    int blocks = per_sm * h->nsm;
    if (max_blocks > 0) blocks = std::min(blocks, max_blocks);
    // SM-resident H-solve: block b keeps rows [b ny / G, (b+1) ny / G) of p
    // plus one halo row on each side in shared memory (floats); taken only
    // where every block owns at least one row and the extra shared memory
    // keeps the blocks this launch needs co-resident on each SM
    // With h_resident = 2, z and r of the H-solve also stay on chip, in
    // tensor memory, when every thread's march chunks fit its 16 slots
    // (tm_slots); the TMEM kernel then runs alone on each SM.
    const bool want_s = P.s_resident != 0;
    P.s_resident = 0;
    if (P.resident) {
        const int want = P.resident;
        P.resident = 0;
        if (h->kind == GADI_STENCIL_2D5 && prec != P_FP64 && vec && blocks <= h->ny &&
            (P.mode == MODE_SOLVE || P.mode == MODE_SOLVE_H)) {
            const long long rows = (h->ny + blocks - 1) / blocks;
            const size_t rs = (size_t)(rows + 2) * (size_t)h->nx * sizeof(float);
            int optin = 0;
            CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
            const size_t rsz = std::max(rs, smem);
            const int elems16 = prec == P_FP32 ? 4 : 8;
            const bool tm = want == 2 && blocks <= h->nsm && tm_slots(h->nx / elems16, h->ny, blocks) <= kTmSlots;
            // the TMEM kernel's CGNR on S also runs resident (MODE_SOLVE) when
            // every block owns two rows or more and p fits with two halo
            // rows on each side
            const size_t rs4 = (size_t)(rows + 4) * (size_t)h->nx * sizeof(float);
            const bool sres = want_s && P.mode == MODE_SOLVE && h->ny / blocks >= 2 && rs4 <= (size_t)optin;
            for (int variant = tm ? 2 : 1; variant >= 1 && !P.resident; --variant) {
                const void *kr = variant == 2 ? kernel_2d5_tm(prec, P.ur_dd) : kernel_2d5_res(prec, P.ur_dd);
                const size_t need = variant == 2 && sres ? std::max(rs4, smem) : rsz;
                if (!kr || need > (size_t)optin) continue;
                CK(cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
                int per_sm_r = 0;
                CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_r, kr, kThreadsHost, need));
                if ((long long)per_sm_r * h->nsm >= blocks && (variant == 1 || per_sm_r == 1)) {
                    P.resident = variant;
                    P.s_resident = variant == 2 && sres;
                    smem = need;
                    k = kr;
                }
            }
        }
    }
    gadi_status s = ensure_ctl(h, blocks, std::max(P.maxit, 1));
    if (s != GADI_OK) return s;
    P.part = h->d_part;
    P.hist = h->d_hist;
    P.ctl = h->d_ctl;
    P.bar = h->d_bar;
    P.abort_flag = h->d_abort;
    CK(cudaMemsetAsync(h->d_bar, 0, 64, st));
    CK(cudaMemsetAsync(h->d_abort, 0, 64, st));
    CK(cudaMemsetAsync(h->d_ctl, 0, sizeof(Ctl), st));
    fill_coef_sets(P);
    void *args[] = {&P};
    CK(cudaLaunchCooperativeKernel(k, dim3(blocks), dim3(kThreadsHost), args, smem, st));
    if (blocks_out) *blocks_out = blocks;
    return GADI_OK;
}

// read back the control block and the abort flag; TIMEOUT if a wait gave up
gadi_status finish(gadi_handle *h, cudaStream_t st)
{
    CK(cudaMemcpyAsync(h->h_ctl, h->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h->h_flag, h->d_abort, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h->h_flag[0]) return GADI_ERR_TIMEOUT;
    return GADI_OK;
}

void fill_base(gadi_handle *h, Params &P, int prec)
{
    std::memset(&P, 0, sizeof P);
    P.kind = h->kind;
    P.sig = h->d_sig;
    P.sig_a = 1.0;
    P.prec = prec;
    P.nx = h->nx;
    P.ny = h->ny;
    P.nz = h->nz;
    P.npts = h->npts;
    P.nelem = h->nelem;
    Coefs &c = P.co;
    c.a_d = h->A.d;
    c.a_e = h->A.e;
    for (int k = 0; k < 6; k++) {
        c.a_c[k] = h->A.c[k];
        c.m_c[k] = h->M.c[k];
        c.n_c[k] = h->N.c[k];
    }
    c.m_d = h->M.d;
    c.n_e = h->N.e;
    if (h->kind == GADI_CSR) {
        P.rowptr = h->d_rowptr;
        P.col = h->d_col;
        P.aval = h->d_aval;
        P.mrowptr = h->d_mrowptr;
        P.mcol = h->d_mcol;
        P.mval_d = h->d_mval;
        P.nval_d = h->d_nval;
    }
}

// inner-solve coefficients for (alpha, omega, prec)
void fill_inner(gadi_handle *h, Params &P, int prec, double alpha, double omega)
{
    Coefs &c = P.co;
    c.h_d = round_us(prec, alpha + h->M.d);
    c.s_d = round_us(prec, alpha);
    c.t_d = c.s_d;
    for (int k = 0; k < 6; k++) {
        c.h_c[k] = round_us(prec, h->M.c[k]);
        c.s_c[k] = round_us(prec, h->N.c[k]);
        c.t_c[k] = -c.s_c[k];
    }
    c.s_e = round_us(prec, h->N.e);
    c.t_e = -c.s_e;
    c.gamma = round_compute(prec, (2.0 - omega) * alpha);
    if (h->kind == GADI_CSR) {
        const size_t eb = elem_bytes(prec), nn = (size_t)h->nnzm;
        P.hval = h->d_opval;
        P.sval = (const char *)h->d_opval + nn * eb;
        P.tval = (const char *)h->d_opval + 2 * nn * eb;
    }
    fill_coef_sets(P);
}

__global__ void k_nonfinite(const double *v, long long n, int *flag)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) {
            atomicExch(flag, 1);
            return;
        }
}

// block 0 never arrives: the other blocks' barrier waits run out
// integer-pipe conversions against the hardware ones (gadi_selftest_convert)
__global__ void k_selftest_convert(const double *in, long long n, unsigned long long *bad)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double d = in[i];
        if (__float_as_uint(f64_to_f32_fast(d)) != __float_as_uint(__double2float_rn(d))) atomicAdd(bad, 1ull);
        if (f64_to_bf16_fast(d) != f64_to_bf16(d)) atomicAdd(bad + 1, 1ull);
        const float g = __uint_as_float((uint32_t)__double_as_longlong(d));
        if (__double_as_longlong(f32_to_f64_fast(g)) != __double_as_longlong((double)g)) atomicAdd(bad + 2, 1ull);
        if (!isnan(g) && f32_to_bf16_cvt(g) != f32_to_bf16(g)) atomicAdd(bad + 3, 1ull);
        // the pair form (two roundings by one instruction): g with the float
        // of the upper 32 bits of d, in both positions of the pair
        const float g2 = __uint_as_float((uint32_t)((unsigned long long)__double_as_longlong(d) >> 32));
        if (!isnan(g) && !isnan(g2)) {
            float a, b;
            f32x2_round_bf16(g, g2, a, b);
            const bool ok1 = __float_as_uint(a) == (uint32_t)f32_to_bf16(g) << 16 &&
                             __float_as_uint(b) == (uint32_t)f32_to_bf16(g2) << 16;
            f32x2_round_bf16(g2, g, a, b);
            const bool ok2 = __float_as_uint(a) == (uint32_t)f32_to_bf16(g2) << 16 &&
                             __float_as_uint(b) == (uint32_t)f32_to_bf16(g) << 16;
            if (!ok1 || !ok2) atomicAdd(bad + 3, 1ull);
        }
    }
}

__global__ void k_barrier_selftest(unsigned long long *counter, int *abort_flag, unsigned long long timeout_ns)
{
    if (blockIdx.x == 0) return;
    GridSync gs;
    gs.counter = counter;
    gs.abort_flag = abort_flag;
    gs.nblocks = gridDim.x;
    gs.timeout_ns = timeout_ns;
    (void)gs.sync();
}

// `iters` grid-wide sums of two FP32 partials, each exactly as the inner
// solves take one (block tree, partial to a slot, grid barrier, every block
// loads all partials); block 0 reports the elapsed %globaltimer time.  The
// partials stay finite (each round feeds a scaled total back in).
__global__ void __launch_bounds__(kThreadsHost, 1)
    k_probe_sync(double *part, unsigned long long *counter, int *abort_flag, int iters, unsigned long long *t_out,
                 float *sink)
{
    GridSync gs;
    gs.counter = counter;
    gs.abort_flag = abort_flag;
    gs.nblocks = gridDim.x;
    const int G = gridDim.x;
    float acc[2] = {(float)threadIdx.x * 1e-3f, 1.0f}, out[2] = {0.f, 0.f};
    int slot = 0;
    if (!gs.sync()) return;
    const unsigned long long t0 = globaltimer_ns();
    for (int i = 0; i < iters; i++) {
        float *pt = reinterpret_cast<float *>(part + (size_t)slot * 2 * G);
        block_partials_write<2, float>(acc, pt, G, blockIdx.x);
        if (!gs.sync()) return;
        grid_partials_sum<2, float>(pt, G, out);
        acc[0] = out[0] * 1e-6f + (float)threadIdx.x * 1e-3f;
        slot ^= 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *t_out = globaltimer_ns() - t0;
        *sink = out[0] + out[1];
    }
}

// FP64 fused multiply-add throughput: 8 independent chains per thread (the
// pipe, not the chain latency, sets the rate), `iters` rounds; the results
// are stored so the chains are not removed
__global__ void __launch_bounds__(kThreadsHost, 1) k_probe_dfma(int iters, double *sink)
{
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = 1.0 + 1e-9 * (threadIdx.x + k);
    const double m = 0.999999999, c = 1e-12 * (blockIdx.x + 1);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) a[k] = fma(a[k], m, c);
    }
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < 8; k++) t += a[k];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

gadi_status check_finite_dev(gadi_handle *h, const double *v, long long n, cudaStream_t st, bool *ok)
{
    CK(cudaMemsetAsync(h->d_flag, 0, sizeof(int), st));
    k_nonfinite<<<std::max(1, h->nsm * 4), 256, 0, st>>>(v, n, h->d_flag);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->h_flag + 1, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *ok = h->h_flag[1] == 0;
    return GADI_OK;
}

bool check_finite_host(const double *v, long long n)
{
    for (long long i = 0; i < n; i++)
        if (!std::isfinite(v[i])) return false;
    return true;
}

__global__ void k_dot(const double *a, const double *b, long long n, double *out)
{
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        s = fma(a[i], b[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}
__global__ void k_scale_copy(const double *a, double s, long long n, double *out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] * s;
}
__global__ void k_init_pw(double *v, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull + 0x1234567ull;
        z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ull;
        v[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0) + 0.5;
    }
}

gadi_status apply_dev(gadi_handle *h, gadi_op op, const double *x, double *y, cudaStream_t st)
{
    Params P;
    fill_base(h, P, P_FP64);
    P.mode = MODE_APPLY;
    P.op = op;
    P.ax_in = x;
    P.ax_out = y;
    P.maxit = 1;
    if (h->kind == GADI_CSR) {
        if (op != GADI_OP_A) {
            P.rowptr = h->d_mrowptr;
            P.col = h->d_mcol;
            P.aval = op == GADI_OP_M ? h->d_mval : (op == GADI_OP_N ? h->d_nval : h->d_atval);
        }
    } else {
        const Stencil &M = h->M, &N = h->N;
        Stencil s{};
        // a per-point T enters A and N with +, A^T with -, M not at all
        P.sig_a = op == GADI_OP_AT ? -1.0 : 1.0;
        if (op == GADI_OP_M) P.sig = nullptr;
        if (op == GADI_OP_A) s = h->A;
        else if (op == GADI_OP_M) s = M;
        else if (op == GADI_OP_N) s = N;
        else { // transpose of the real (block) form: M - N
            s.d = M.d - N.d;
            for (int k = 0; k < 6; k++) s.c[k] = M.c[k] - N.c[k];
            s.e = M.e - N.e;
        }
        P.co.a_d = s.d;
        P.co.a_e = s.e;
        for (int k = 0; k < 6; k++) P.co.a_c[k] = s.c[k];
    }
    gadi_status r = launch(h, P_FP64, P, 0, st, nullptr);
    if (r != GADI_OK) return r;
    return finish(h, st);
}

gadi_status opts_check(const gadi_opts &o)
{
    if (!(o.tol_h >= 0) || !(o.tol_s >= 0) || o.maxit_inner < 0 || o.inner_stag < 0 || o.outer_stag_window < 0)
        return GADI_ERR_INVALID;
    if (o.h_resident < 0 || o.h_resident > 2) return GADI_ERR_INVALID;
    if (o.s_resident != 0 && o.s_resident != 1) return GADI_ERR_INVALID;
    if (o.u_r != GADI_FP64 && o.u_r != GADI_FP64X2) return GADI_ERR_INVALID;
    if (o.backward_err < 0) return GADI_ERR_INVALID;
    if (o.batch_interleave != 0 && o.batch_interleave != 1) return GADI_ERR_INVALID;
    return GADI_OK;
}

} // namespace

// ==========================================================================
// public API
// ==========================================================================
extern "C" {

void gadi_opts_default(gadi_opts *o, gadi_prec u_low)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->tol_h = o->tol_s = (u_low == GADI_BF16) ? 1e-2 : 1e-3;
    o->maxit_inner = 1000;
    o->inner_stag = 10;
    o->outer_stag_window = 50;
    o->s_pointwise = 1;
    o->stream = nullptr;
    o->max_blocks = 0;
    o->hist = nullptr;
    o->batch_group = 0;
    o->alpha_restarts = 0;
    // tensor-memory z and r measured faster for FP32 (CG on H at 2048^2:
    // 12.0 vs 13.2 us per iteration) and slower for BF16 (17.6 vs 16.3)
    o->h_resident = (u_low == GADI_BF16) ? 1 : 2;
    o->u_r = GADI_FP64;
    o->s_resident = 1;
    o->batch_interleave = 0;
}

const char *gadi_last_error(void) { return g_last_error; }

} // extern "C"

void gadi::record_error(const char *msg) { std::snprintf(g_last_error, sizeof g_last_error, "%s", msg); }

extern "C" {

const char *gadi_status_str(gadi_status s)
{
    switch (s) {
    case GADI_OK: return "GADI_OK";
    case GADI_NOT_CONVERGED: return "GADI_NOT_CONVERGED";
    case GADI_STAGNATED: return "GADI_STAGNATED";
    case GADI_DIVERGED: return "GADI_DIVERGED";
    case GADI_ERR_INVALID: return "GADI_ERR_INVALID";
    case GADI_ERR_NONFINITE: return "GADI_ERR_NONFINITE";
    case GADI_ERR_CUDA: return "GADI_ERR_CUDA";
    case GADI_ERR_OOM: return "GADI_ERR_OOM";
    case GADI_ERR_TIMEOUT: return "GADI_ERR_TIMEOUT";
    case GADI_ERR_UNSUPPORTED: return "GADI_ERR_UNSUPPORTED";
    }
    return "GADI_UNKNOWN_STATUS";
}

gadi_status gadi_create(const gadi_problem *p, gadi_splitting split, gadi_handle **out)
{
    if (!out) return GADI_ERR_INVALID;
    *out = nullptr;
    if (!p || split != GADI_SPLIT_HSS) return GADI_ERR_INVALID;
    if (p->kind < GADI_STENCIL_2D5 || p->kind > GADI_CSR) return GADI_ERR_INVALID;
    gadi_handle *h = new (std::nothrow) gadi_handle();
    if (!h) return GADI_ERR_OOM;
    h->kind = p->kind;
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
        delete h;
        return GADI_ERR_CUDA;
    }
    gadi_status st = GADI_OK;
    if (p->kind != GADI_CSR) {
        if (p->nx <= 0 || p->ny <= 0 || (p->kind == GADI_STENCIL_3D7 && p->nz <= 0)) st = GADI_ERR_INVALID;
        for (int k = 0; k < 3; k++)
            if (!std::isfinite(p->beta[k])) st = GADI_ERR_NONFINITE;
        if (!std::isfinite(p->kappa) || !std::isfinite(p->sigma) || !std::isfinite(p->h)) st = GADI_ERR_NONFINITE;
        if (st == GADI_OK && p->kappa < 0) st = GADI_ERR_INVALID; // M must stay positive definite
        if (st == GADI_OK) {
            h->nx = p->nx;
            h->ny = p->ny;
            h->nz = p->kind == GADI_STENCIL_3D7 ? p->nz : 1;
            h->npts = (long long)h->nx * h->ny * h->nz;
            h->nelem = h->kind == GADI_COMPLEX_2D5 ? 2 * h->npts : h->npts;
            // the kernels index work units and rows with 32-bit integers
            if (h->nelem > (1ll << 31) - (1ll << 24)) st = GADI_ERR_INVALID;
            h->h = p->h > 0 ? p->h : 1.0 / (p->nx + 1);
            for (int k = 0; k < 3; k++) h->beta[k] = p->beta[k];
            h->kappa = p->kappa;
            h->sigma = p->sigma;
            stencil_coefs(h);
        }
        if (st == GADI_OK && p->kind == GADI_COMPLEX_2D5 && p->sigma_pt) {
            for (long long i = 0; i < h->npts; i++)
                if (!std::isfinite(p->sigma_pt[i])) st = GADI_ERR_NONFINITE;
            if (st == GADI_OK) {
                const size_t bytes = sizeof(double) * (size_t)h->npts;
                if (cudaMalloc(&h->d_sig, bytes) != cudaSuccess) st = GADI_ERR_OOM;
                else if (cudaMemcpy(h->d_sig, p->sigma_pt, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
                    st = GADI_ERR_CUDA;
            }
        }
    } else {
        const int n = p->n;
        if (n <= 0 || !p->rowptr || !p->col || !p->val) st = GADI_ERR_INVALID;
        if (st == GADI_OK && (p->rowptr[0] != 0)) st = GADI_ERR_INVALID;
        if (st == GADI_OK)
            for (int i = 0; i < n; i++)
                if (p->rowptr[i + 1] < p->rowptr[i]) st = GADI_ERR_INVALID;
        const int nnz = st == GADI_OK ? p->rowptr[n] : 0;
        if (st == GADI_OK)
            for (int k = 0; k < nnz; k++) {
                if (p->col[k] < 0 || p->col[k] >= n) st = GADI_ERR_INVALID;
                if (!std::isfinite(p->val[k])) st = GADI_ERR_NONFINITE;
            }
        if (st == GADI_OK) {
            h->npts = h->nelem = n;
            h->nx = n;
            h->ny = h->nz = 1;
            h->nnz = nnz;
            // M = (A + A^T)/2, N = (A - A^T)/2 on the union pattern plus the
            // diagonal, columns sorted (dense row scatter, one row at a time)
            std::vector<std::vector<std::pair<int, double>>> at(n);
            for (int i = 0; i < n; i++)
                for (int k = p->rowptr[i]; k < p->rowptr[i + 1]; k++) at[p->col[k]].push_back({i, p->val[k]});
            std::vector<double> ra(n, 0.0), rt(n, 0.0);
            std::vector<char> mark(n, 0);
            std::vector<int> cols;
            h->h_mrowptr.assign(n + 1, 0);
            for (int i = 0; i < n; i++) {
                cols.clear();
                auto touch = [&](int j) {
                    if (!mark[j]) {
                        mark[j] = 1;
                        cols.push_back(j);
                    }
                };
                touch(i);
                for (int k = p->rowptr[i]; k < p->rowptr[i + 1]; k++) {
                    touch(p->col[k]);
                    ra[p->col[k]] += p->val[k];
                }
                for (auto &e : at[i]) {
                    touch(e.first);
                    rt[e.first] += e.second;
                }
                std::sort(cols.begin(), cols.end());
                for (int j : cols) {
                    h->h_mcol.push_back(j);
                    h->h_mval.push_back((ra[j] + rt[j]) * 0.5);
                    h->h_nval.push_back((ra[j] - rt[j]) * 0.5);
                    ra[j] = rt[j] = 0.0;
                    mark[j] = 0;
                }
                h->h_mrowptr[i + 1] = (int)h->h_mcol.size();
            }
            h->nnzm = (int)h->h_mcol.size();
            std::vector<double> atv(h->nnzm);
            for (int k = 0; k < h->nnzm; k++) atv[k] = h->h_mval[k] - h->h_nval[k];
            auto up = [&](void **d, const void *src, size_t bytes) -> bool {
                if (cudaMalloc(d, bytes ? bytes : 16) != cudaSuccess) return false;
                return bytes == 0 || cudaMemcpy(*d, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
            };
            bool ok = up((void **)&h->d_rowptr, p->rowptr, sizeof(int) * (n + 1)) &&
                      up((void **)&h->d_col, p->col, sizeof(int) * nnz) &&
                      up((void **)&h->d_aval, p->val, sizeof(double) * nnz) &&
                      up((void **)&h->d_mrowptr, h->h_mrowptr.data(), sizeof(int) * (n + 1)) &&
                      up((void **)&h->d_mcol, h->h_mcol.data(), sizeof(int) * h->nnzm) &&
                      up((void **)&h->d_mval, h->h_mval.data(), sizeof(double) * h->nnzm) &&
                      up((void **)&h->d_nval, h->h_nval.data(), sizeof(double) * h->nnzm) &&
                      up((void **)&h->d_atval, atv.data(), sizeof(double) * h->nnzm);
            if (!ok) st = GADI_ERR_OOM;
        }
    }
    if (st == GADI_OK) st = ensure_ctl(h, 1, 1);
    if (st != GADI_OK) {
        gadi_destroy(h);
        return st;
    }
    *out = h;
    return GADI_OK;
}

void gadi_destroy(gadi_handle *h)
{
    if (!h) return;
    void *dev[] = {h->d_rowptr, h->d_col, h->d_mrowptr, h->d_mcol, h->d_aval, h->d_mval, h->d_nval,
                   h->d_atval, h->d_opval, h->d_ws, h->d_part, h->d_hist, h->d_ctl, h->d_bar,
                   h->d_abort, h->d_flag, h->d_stage, h->d_pw, h->d_sig, h->d_acc};
    for (void *p : dev)
        if (p) cudaFree(p);
    if (h->h_ctl) cudaFreeHost(h->h_ctl);
    if (h->h_flag) cudaFreeHost(h->h_flag);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    delete h;
}

} // extern "C"

namespace {
gadi_status solve_once(gadi_handle *h, const double *b, double *x, double alpha, double omega,
                       gadi_prec u_high, gadi_prec u_low, double tol, int maxit, const gadi_opts *opts,
                       gadi_stats *stats)
{
    if (!h || !b || !x) return GADI_ERR_INVALID;
    if (!std::isfinite(alpha) || !std::isfinite(omega) || std::isnan(tol)) return GADI_ERR_NONFINITE;
    if (!(alpha > 0) || !(omega >= 0 && omega < 2) || u_high != GADI_FP64 || !(tol >= 0) || maxit < 0)
        return GADI_ERR_INVALID;
    if (u_low != GADI_FP64 && u_low != GADI_FP32 && u_low != GADI_BF16) return GADI_ERR_INVALID;
    gadi_opts o;
    if (opts) o = *opts;
    else gadi_opts_default(&o, u_low);
    gadi_status s = opts_check(o);
    if (s != GADI_OK) return s;
    const int prec = (int)u_low;
    cudaStream_t st = (cudaStream_t)o.stream;
    const long long m = h->nelem;
    const size_t vb = sizeof(double) * (size_t)m;

    // stage host vectors
    const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
    if (!bdev || !xdev) {
        if (!h->d_stage) CK(cudaMalloc(&h->d_stage, 2 * vb));
    }
    if (!bdev && !check_finite_host(b, m)) return GADI_ERR_NONFINITE;
    if (!xdev && !check_finite_host(x, m)) return GADI_ERR_NONFINITE;
    const double *db = bdev ? b : h->d_stage;
    double *dx = xdev ? x : h->d_stage + m;
    if (!bdev) CK(cudaMemcpyAsync((void *)db, b, vb, cudaMemcpyHostToDevice, st));
    if (!xdev) CK(cudaMemcpyAsync(dx, x, vb, cudaMemcpyHostToDevice, st));
    if (bdev || xdev) {
        bool ok = true;
        if (bdev && (s = check_finite_dev(h, b, m, st, &ok)) != GADI_OK) return s;
        if (!ok) return GADI_ERR_NONFINITE;
        if (xdev && (s = check_finite_dev(h, x, m, st, &ok)) != GADI_OK) return s;
        if (!ok) return GADI_ERR_NONFINITE;
    }

    Work w;
    if ((s = ensure_ws(h, prec, &w)) != GADI_OK) return s;
    if (h->kind == GADI_CSR && (s = ensure_csr_ops(h, prec, alpha)) != GADI_OK) return s;
    Params P;
    fill_base(h, P, prec);
    fill_inner(h, P, prec, alpha, omega);
    P.mode = MODE_SOLVE;
    P.b = db;
    P.x = dx;
    set_work(P, w);
    P.tol = tol;
    P.tol_h = o.tol_h;
    P.tol_s = o.tol_s;
    P.maxit = maxit;
    P.maxit_inner = o.maxit_inner;
    P.inner_stag = o.inner_stag;
    P.outer_win = o.outer_stag_window;
    P.pointwise = o.s_pointwise;
    P.resident = o.h_resident;
    P.s_resident = o.s_resident; // a request; launch() keeps it only where it applies
    P.ur_dd = o.u_r == GADI_FP64X2;
    CK(cudaEventRecord(h->ev0, st));
    int blocks = 0;
    if ((s = launch(h, prec, P, o.max_blocks, st, &blocks)) != GADI_OK) return s;
    CK(cudaEventRecord(h->ev1, st));
    if ((s = finish(h, st)) != GADI_OK) return s;
    const Ctl c = *h->h_ctl;
    if (c.x_in_x1) CK(cudaMemcpyAsync(dx, w.x1, vb, cudaMemcpyDeviceToDevice, st));
    if (!xdev) CK(cudaMemcpyAsync(x, dx, vb, cudaMemcpyDeviceToHost, st));
    if (o.hist) CK(cudaMemcpyAsync(o.hist, h->d_hist, sizeof(double) * (size_t)(c.outer_its + 1),
                                   cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    if (stats) {
        stats->outer_its = c.outer_its;
        stats->inner_its_h = c.inner_h;
        stats->inner_its_s = c.inner_s;
        stats->relres = c.relres;
        stats->r0_norm = c.r0;
        stats->seconds = ms * 1e-3;
        stats->status = c.status;
        stats->blocks = blocks;
        stats->alpha = alpha;
        stats->restarts = 0;
        stats->h_resident = P.resident;
        stats->s_resident = P.s_resident;
        stats->backward_err = -1.0;
    }
    return (gadi_status)c.status;
}

// ||v||_2 of an FP64 vector in host or device memory (device: a grid-stride
// dot on the handle's stream)
gadi_status vec_norm2(gadi_handle *h, const double *v, long long m, cudaStream_t st, double *out)
{
    if (!is_device_ptr(v)) {
        double s = 0.0;
        for (long long i = 0; i < m; i++) s = std::fma(v[i], v[i], s);
        *out = std::sqrt(s);
        return GADI_OK;
    }
    if (!h->d_acc) CK(cudaMalloc(&h->d_acc, 2 * sizeof(double)));
    CK(cudaMemsetAsync(h->d_acc, 0, sizeof(double), st));
    k_dot<<<std::max(1, h->nsm * 4), 256, 0, st>>>(v, v, m, h->d_acc);
    CK(cudaGetLastError());
    double hs = 0.0;
    CK(cudaMemcpyAsync(&hs, h->d_acc, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *out = std::sqrt(hs);
    return GADI_OK;
}

// closed-form spectra of the stencil classes (Sec. 4.3, the condition check)
bool stencil_spectra(const gadi_problem *p, double *lmin, double *lmax, double *nnorm)
{
    if (!p || p->kind == GADI_CSR || p->kind < 0 || p->kind > GADI_CSR) return false;
    if (p->nx <= 0 || p->ny <= 0 || (p->kind == GADI_STENCIL_3D7 && p->nz <= 0)) return false;
    const double h = p->h > 0 ? p->h : 1.0 / (p->nx + 1);
    const int dims = p->kind == GADI_STENCIL_3D7 ? 3 : 2;
    const int n[3] = {p->nx, p->ny, p->nz};
    const double pi = 3.14159265358979323846;
    double lo = 0, hi = 0, nn = 0;
    for (int d = 0; d < dims; d++) {
        const double t = pi / (2.0 * (n[d] + 1));
        lo += 4.0 * std::sin(t) * std::sin(t); // 1D Dirichlet Laplacian 2 - 2 cos(j pi/(n+1))
        hi += 4.0 * std::cos(t) * std::cos(t);
        if (p->kind != GADI_COMPLEX_2D5) nn += 2.0 * std::fabs(p->beta[d] * h / 2.0) * std::cos(2.0 * t);
    }
    lo += p->kappa;
    hi += p->kappa;
    if (p->kind == GADI_COMPLEX_2D5) {
        nn = std::fabs(p->sigma);
        if (p->sigma_pt) {
            nn = 0.0;
            for (long long i = 0; i < (long long)p->nx * p->ny; i++) nn = std::max(nn, std::fabs(p->sigma_pt[i]));
        }
    }
    *lmin = lo;
    *lmax = hi;
    *nnorm = nn;
    return true;
}
double unit_roundoff(int prec) { return prec == P_BF16 ? 3.91e-3 : (prec == P_FP32 ? 5.96e-8 : 1.11e-16); }

// eq. (3.2): ||r|| / (||A||_2 ||x|| + ||b||) with r_norm the solve's final
// FP64 residual norm; ||A||_2 from o.backward_err power-iteration steps, kept
// by the handle for later solves with the same step count
gadi_status backward_error(gadi_handle *h, const double *b, const double *x, double r_norm, const gadi_opts &o,
                           double *out)
{
    cudaStream_t st = (cudaStream_t)o.stream;
    if (h->anorm < 0 || h->anorm_iters != o.backward_err) {
        double an = 0.0;
        const gadi_status e = gadi_norm2_estimate(h, o.backward_err, &an, o.stream);
        if (e != GADI_OK) return e;
        h->anorm = an;
        h->anorm_iters = o.backward_err;
    }
    double xn = 0.0, bn = 0.0;
    gadi_status e = vec_norm2(h, x, h->nelem, st, &xn);
    if (e == GADI_OK) e = vec_norm2(h, b, h->nelem, st, &bn);
    if (e != GADI_OK) return e;
    const double den = h->anorm * xn + bn;
    *out = den > 0 ? r_norm / den : 0.0;
    return GADI_OK;
}
} // namespace

extern "C" {

gadi_status gadi_selftest_convert(const double *in, long long n, long long *mismatches)
{
    if (!in || !mismatches || n < 0) return GADI_ERR_INVALID;
    unsigned long long *d_bad = nullptr, hb[4] = {0, 0, 0, 0};
    CK(cudaMalloc(&d_bad, sizeof hb));
    cudaError_t e = cudaMemset(d_bad, 0, sizeof hb);
    if (e == cudaSuccess && n > 0) {
        const long long nb = std::min<long long>((n + 255) / 256, 4096);
        k_selftest_convert<<<(unsigned)nb, 256>>>(in, n, d_bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(hb, d_bad, sizeof hb, cudaMemcpyDeviceToHost);
    cudaFree(d_bad);
    if (e != cudaSuccess) return cuda_err(e, "gadi_selftest_convert", __LINE__);
    for (int k = 0; k < 4; k++) mismatches[k] = (long long)hb[k];
    return GADI_OK;
}

gadi_status gadi_selftest_barrier(int nblocks, double timeout_ms)
{
    if (nblocks < 2 || !(timeout_ms > 0) || timeout_ms > 10000.0) return GADI_ERR_INVALID;
    int dev = 0, nsm = 0, per_sm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_barrier_selftest, 32, 0));
    if (nblocks > per_sm * nsm) return GADI_ERR_INVALID;
    unsigned long long *buf = nullptr;
    CK(cudaMalloc(&buf, 128));
    gadi_status st = GADI_OK;
    int hab = 0;
    unsigned long long *counter = buf;
    int *abort_flag = (int *)(buf + 8);
    unsigned long long tns = (unsigned long long)(timeout_ms * 1e6);
    void *args[] = {&counter, &abort_flag, &tns};
    cudaError_t e = cudaMemset(buf, 0, 128);
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel((const void *)k_barrier_selftest, dim3(nblocks), dim3(32), args, 0, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&hab, abort_flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) st = cuda_err(e, "gadi_selftest_barrier", __LINE__);
    else if (hab) st = GADI_ERR_TIMEOUT;
    cudaFree(buf);
    return st;
}

gadi_status gadi_stencil_coefs(const gadi_problem *p, gadi_op op, double *coef)
{
    if (!p || !coef || p->kind == GADI_CSR || p->kind < GADI_STENCIL_2D5 || p->kind > GADI_CSR) return GADI_ERR_INVALID;
    if (op < GADI_OP_A || op > GADI_OP_AT) return GADI_ERR_INVALID;
    if (p->nx <= 0 || !(p->kappa >= 0) || !std::isfinite(p->h)) return GADI_ERR_INVALID;
    gadi_handle h;
    h.kind = p->kind;
    h.nx = p->nx;
    h.h = p->h > 0 ? p->h : 1.0 / (p->nx + 1);
    for (int k = 0; k < 3; k++) h.beta[k] = p->beta[k];
    h.kappa = p->kappa;
    h.sigma = p->sigma;
    stencil_coefs(&h);
    const Stencil &M = h.M, &N = h.N;
    Stencil s{};
    if (op == GADI_OP_A) s = h.A;
    else if (op == GADI_OP_M) s = M;
    else if (op == GADI_OP_N) s = N;
    else {
        s.d = M.d - N.d;
        for (int k = 0; k < 6; k++) s.c[k] = M.c[k] - N.c[k];
        s.e = M.e - N.e;
    }
    coef[0] = s.d;
    for (int k = 0; k < 6; k++) coef[1 + k] = s.c[k];
    coef[7] = s.e;
    return GADI_OK;
}

gadi_status gadi_probe_sync(int nblocks, int iters, double *us_per_sum)
{
    if (!us_per_sum || iters <= 0 || iters > 1000000) return GADI_ERR_INVALID;
    int dev = 0, nsm = 0, per_sm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_probe_sync, kThreadsHost, 0));
    if (nblocks == 0) nblocks = nsm;
    if (nblocks < 1 || nblocks > per_sm * nsm) return GADI_ERR_INVALID;
    // partials (2 slots x 2 values x nblocks doubles), counter, abort flag,
    // elapsed time, sink
    const size_t part_bytes = sizeof(double) * 4 * (size_t)nblocks;
    char *buf = nullptr;
    CK(cudaMalloc(&buf, part_bytes + 256));
    double *part = (double *)buf;
    unsigned long long *counter = (unsigned long long *)(buf + part_bytes);
    int *abort_flag = (int *)(buf + part_bytes + 64);
    unsigned long long *t_out = (unsigned long long *)(buf + part_bytes + 128);
    float *sink = (float *)(buf + part_bytes + 192);
    void *args[] = {&part, &counter, &abort_flag, &iters, &t_out, &sink};
    unsigned long long tns = 0;
    int hab = 0;
    gadi_status st = GADI_OK;
    cudaError_t e = cudaMemset(buf, 0, part_bytes + 256);
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel((const void *)k_probe_sync, dim3(nblocks), dim3(kThreadsHost), args, 0, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&tns, t_out, sizeof tns, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&hab, abort_flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) st = cuda_err(e, "gadi_probe_sync", __LINE__);
    else if (hab) st = GADI_ERR_TIMEOUT;
    else *us_per_sum = (double)tns * 1e-3 / iters;
    cudaFree(buf);
    return st;
}

gadi_status gadi_probe_fp64(int iters, double *gops, double *sm_ops_per_clk)
{
    if (!gops || iters <= 0 || iters > 10000000) return GADI_ERR_INVALID;
    int dev = 0, nsm = 0, clk_khz = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev));
    double *sink = nullptr;
    CK(cudaMalloc(&sink, sizeof(double) * (size_t)nsm * kThreadsHost));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gadi_status st = GADI_OK;
    float ms = 0.f;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        k_probe_dfma<<<nsm, kThreadsHost>>>(iters / 10 + 1, sink); // warm-up (clocks, code)
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) {
        k_probe_dfma<<<nsm, kThreadsHost>>>(iters, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) st = cuda_err(e, "gadi_probe_fp64", __LINE__);
    else {
        const double ops = 8.0 * iters * (double)nsm * kThreadsHost;
        *gops = ops / (ms * 1e-3) / 1e9;
        if (sm_ops_per_clk) *sm_ops_per_clk = ops / (ms * 1e-3) / nsm / (clk_khz * 1e3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return st;
}

gadi_status gadi_condition_numbers(const gadi_problem *prob, double alpha, double *kappa_h, double *kappa_s)
{
    if (!prob || !kappa_h || !kappa_s || !(alpha > 0) || !std::isfinite(alpha)) return GADI_ERR_INVALID;
    if (prob->kind == GADI_CSR) return GADI_ERR_UNSUPPORTED;
    double lo, hi, nn;
    if (!stencil_spectra(prob, &lo, &hi, &nn)) return GADI_ERR_INVALID;
    *kappa_h = (alpha + hi) / (alpha + lo);
    *kappa_s = std::sqrt(alpha * alpha + nn * nn) / alpha;
    return GADI_OK;
}

gadi_status gadi_select_alpha(const gadi_problem *prob, double alpha0, gadi_prec u_low, double tau,
                              double *alpha_out)
{
    if (!alpha_out || !(tau > 0)) return GADI_ERR_INVALID;
    if (u_low != GADI_FP64 && u_low != GADI_FP32 && u_low != GADI_BF16) return GADI_ERR_INVALID;
    double a = alpha0;
    for (int k = 0; k <= 60; k++, a *= 2.0) {
        double kh, ks;
        gadi_status st = gadi_condition_numbers(prob, a, &kh, &ks);
        if (st != GADI_OK) return st;
        if (kh * ks * unit_roundoff((int)u_low) < tau) {
            *alpha_out = a;
            return GADI_OK;
        }
    }
    return GADI_ERR_INVALID;
}

gadi_status gadi_solve(gadi_handle *h, const double *b, double *x, double alpha, double omega,
                       gadi_prec u_high, gadi_prec u_low, double tol, int maxit, const gadi_opts *opts,
                       gadi_stats *stats)
{
    gadi_opts o;
    if (opts) o = *opts;
    else gadi_opts_default(&o, u_low);
    gadi_stats st1;
    gadi_status s = solve_once(h, b, x, alpha, omega, u_high, u_low, tol, maxit, &o, &st1);
    if (s < 0 || o.alpha_restarts <= 0 || (s != GADI_STAGNATED && s != GADI_DIVERGED)) {
        if (s >= 0 && o.backward_err > 0) {
            const gadi_status e = backward_error(h, b, x, st1.relres * st1.r0_norm, o, &st1.backward_err);
            if (e != GADI_OK) return e;
        }
        if (stats) *stats = st1;
        return s;
    }
    // Sec. 4.3: on stagnation or divergence, a larger alpha and a new run -- from the last iterate,
    // with the tolerance kept relative to the first residual norm
    gadi_stats acc = st1;
    const double r0 = st1.r0_norm;
    double a = alpha, rel = st1.relres;
    int its_left = maxit - st1.outer_its;
    for (int k = 0; k < o.alpha_restarts && (s == GADI_STAGNATED || s == GADI_DIVERGED) && its_left > 0; k++) {
        a *= 2.0;
        if (!(rel == rel) || std::isinf(rel)) return s; // no finite iterate to continue from
        const double tol_k = r0 > 0 && rel > 0 ? tol / rel : tol;
        gadi_opts ok = o;
        ok.hist = nullptr;
        gadi_stats sk;
        s = solve_once(h, b, x, a, omega, u_high, u_low, tol_k, its_left, &ok, &sk);
        if (s < 0) return s;
        rel = rel * sk.relres;
        its_left -= sk.outer_its;
        acc.outer_its += sk.outer_its;
        acc.inner_its_h += sk.inner_its_h;
        acc.inner_its_s += sk.inner_its_s;
        acc.seconds += sk.seconds;
        acc.restarts = k + 1;
        acc.alpha = a;
        acc.status = s;
    }
    acc.relres = rel;
    if (s >= 0 && o.backward_err > 0) {
        const gadi_status e = backward_error(h, b, x, rel * r0, o, &acc.backward_err);
        if (e != GADI_OK) return e;
    }
    if (stats) *stats = acc;
    return s;
}

} // extern "C"

namespace {

// ---------------------------------------------------------------------------
// batched solve: size classes, group sizes and one launch
// ---------------------------------------------------------------------------
// A group layout: the groups' sizes and classes in block order.
struct BatchLayout {
    std::vector<int> gsize, gclass; // per group
    int blocks = 0;
};

// Device buffers of one batched launch, freed on every way out.
struct DevBuf {
    void *p = nullptr;
    ~DevBuf()
    {
        if (p) cudaFree(p);
    }
};

// One cooperative launch of the batched kernel over `units` (already filled
// but for the work pointers), classes given by class_begin / order, groups by
// `lay`.  Per-unit control blocks, start and end times come back in ctl, t0,
// t1.  timed_s (nullable): device time of the launch (events on h0).
gadi_status run_batch(gadi_handle *h0, const void *k, size_t smem, std::vector<Params> &units,
                      const std::vector<int> &class_begin, const std::vector<int> &order, const BatchLayout &lay,
                      long long max_n, int prec, int hist_len, cudaStream_t st, std::vector<Ctl> &ctl,
                      std::vector<unsigned long long> &t0, std::vector<unsigned long long> &t1, float *timed_ms,
                      int nr = 1, const std::vector<int> *gmin = nullptr, const std::vector<int> *gmax = nullptr)
{
    // nr = 4: units of four interleaved right-hand sides (gadi_batched4_kernel):
    // 4x the vectors, a third FP64 work vector, 4 control blocks and 4
    // histories per unit, 16 partial sums per block
    const int nunits = (int)units.size(), ngroups = (int)lay.gsize.size(), nclasses = (int)class_begin.size() - 1;
    std::vector<int> block_group(lay.blocks), group_first(ngroups);
    for (int g = 0, b0 = 0; g < ngroups; b0 += lay.gsize[g], g++) {
        group_first[g] = b0;
        for (int j = 0; j < lay.gsize[g]; j++) block_group[b0 + j] = g;
    }
    const size_t slab = align256((size_t)max_n * nr * elem_bytes(prec)), slab_d = align256((size_t)max_n * nr * 8);
    const size_t gwork = (nr == 1 ? 1 : 3) * slab_d + 6 * slab;
    const size_t nctl = (size_t)nunits * nr;
    // one table buffer: block_group, group_first, group_size, group_class,
    // class_begin, order, queues (32 ints a class), group_unit (32 a group)
    const size_t nint = (size_t)lay.blocks + 3 * (size_t)ngroups + (nclasses + 1) + 2 * (size_t)nclasses + nunits +
                        32 * (size_t)nclasses + 32 * (size_t)ngroups;
    std::vector<int> tab(nint, 0);
    size_t off = 0;
    auto put = [&](const std::vector<int> &v) {
        const size_t at = off;
        std::copy(v.begin(), v.end(), tab.begin() + (long)off);
        off += v.size();
        return at;
    };
    const size_t o_bg = put(block_group), o_gf = put(group_first), o_gs = put(lay.gsize), o_gc = put(lay.gclass);
    // the group sizes that may take each class's units (all, unless given)
    const std::vector<int> lo = gmin ? *gmin : std::vector<int>(nclasses, 1);
    const std::vector<int> hi = gmax ? *gmax : std::vector<int>(nclasses, 1 << 30);
    const size_t o_cb = put(class_begin), o_lo = put(lo), o_hi = put(hi), o_or = put(order);
    const size_t o_q = off, o_gu = off + 32 * (size_t)nclasses;
    DevBuf bu, bt, bw, bp, bb, bh, bc, btm;
    CK(cudaMalloc(&bu.p, sizeof(Params) * (size_t)nunits));
    CK(cudaMalloc(&bt.p, sizeof(int) * nint));
    CK(cudaMalloc(&bw.p, gwork * (size_t)ngroups));
    CK(cudaMalloc(&bp.p, sizeof(double) * 4 * nr * (size_t)lay.blocks));
    CK(cudaMalloc(&bb.p, sizeof(unsigned long long) * 8 * (size_t)ngroups + 64));
    CK(cudaMalloc(&bh.p, sizeof(double) * (size_t)hist_len * nr * ngroups));
    CK(cudaMalloc(&bc.p, sizeof(Ctl) * nctl));
    CK(cudaMalloc(&btm.p, sizeof(unsigned long long) * 2 * (size_t)nunits));
    CK(cudaMemcpyAsync(bu.p, units.data(), sizeof(Params) * (size_t)nunits, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(bt.p, tab.data(), sizeof(int) * nint, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(bb.p, 0, sizeof(unsigned long long) * 8 * (size_t)ngroups + 64, st));
    CK(cudaMemsetAsync(bc.p, 0, sizeof(Ctl) * nctl, st));
    const int *ti = (const int *)bt.p;
    BatchParams B;
    std::memset(&B, 0, sizeof B);
    B.units = (Params *)bu.p;
    B.nunits = nunits;
    B.ngroups = ngroups;
    B.nclasses = nclasses;
    B.block_group = ti + o_bg;
    B.group_first = ti + o_gf;
    B.group_size = ti + o_gs;
    B.group_class = ti + o_gc;
    B.class_begin = ti + o_cb;
    B.class_gmin = ti + o_lo;
    B.class_gmax = ti + o_hi;
    B.order = ti + o_or;
    B.queue = (int *)bt.p + o_q;
    B.group_unit = (int *)bt.p + o_gu;
    B.work = (char *)bw.p;
    B.group_work_bytes = gwork;
    B.slab_bytes = slab;
    B.slab_d_bytes = slab_d;
    B.part = (double *)bp.p;
    B.bar = (unsigned long long *)bb.p;
    B.abort_flag = (int *)((unsigned long long *)bb.p + 8 * (size_t)ngroups);
    B.hist = (double *)bh.p;
    B.hist_len = hist_len;
    B.ctl = (Ctl *)bc.p;
    B.t0 = (unsigned long long *)btm.p;
    B.t1 = B.t0 + nunits;
    void *args[] = {&B};
    CK(cudaEventRecord(h0->ev0, st));
    CK(cudaLaunchCooperativeKernel(k, dim3(lay.blocks), dim3(kThreadsHost), args, smem, st));
    CK(cudaEventRecord(h0->ev1, st));
    ctl.assign(nctl, Ctl{});
    t0.assign(nunits, 0);
    t1.assign(nunits, 0);
    int hab = 0;
    CK(cudaMemcpyAsync(ctl.data(), bc.p, sizeof(Ctl) * nctl, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(t0.data(), btm.p, sizeof(unsigned long long) * (size_t)nunits, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(t1.data(), B.t1, sizeof(unsigned long long) * (size_t)nunits, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&hab, B.abort_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (timed_ms) CK(cudaEventElapsedTime(timed_ms, h0->ev0, h0->ev1));
    if (hab) return GADI_ERR_TIMEOUT;
    return GADI_OK;
}

// Group sizes the tuner tries
constexpr int kTuneSizes[] = {1, 2, 4, 8, 16, 32, 64};
// outer iterations of the two timed trials per size: the cost per outer
// iteration is taken from their difference, so it is that of the solve's
// later iterations (the first ones, from x = 0, need fewer inner steps)
constexpr int kTuneOuterA = 8, kTuneOuterB = 24;

// measured device seconds per outer iteration of one unit of a system class
// on a group of s blocks, by (grid, precision, residual, inner tolerances,
// blocks available); kept for the life of the process
std::mutex g_tune_mu;
std::map<std::vector<long long>, std::vector<double>> g_tune;

// the key: grid, precision, options, blocks, and the class's alpha values
// (alpha sets the inner iteration counts, hence the cost per outer iteration)
// The resident H-solve on a group of s blocks: block b owns rows [b ny / s,
// (b+1) ny / s) and keeps p of those rows plus a halo row on each side in
// shared memory as floats.  A group may take a unit if each block owns a row
// and its share fits the opt-in shared memory.
size_t res_smem(long long nx, long long ny, int s)
{
    const long long rows = (ny + s - 1) / s;
    return (size_t)(rows + 2) * (size_t)nx * sizeof(float);
}
bool res_allowed(long long nx, long long ny, int s, int optin)
{
    return s <= ny && res_smem(nx, ny, s) <= (size_t)optin;
}

std::vector<long long> tune_key(const gadi_handle *h, int prec, const gadi_opts &o, int total,
                                const std::vector<double> &alphas)
{
    long long th, ts;
    std::memcpy(&th, &o.tol_h, 8);
    std::memcpy(&ts, &o.tol_s, 8);
    std::vector<long long> k = {h->nx, h->ny, prec, o.u_r, th, ts, o.maxit_inner, o.inner_stag, total};
    for (double a : alphas) {
        long long b;
        std::memcpy(&b, &a, 8);
        k.push_back(b);
    }
    return k;
}

// Time outer iterations of the units of a class on groups of each candidate
// size s, with the whole grid busy: total / s groups each run a copy of one of
// the class's units (tol 0, own x), so the trial sees the L2 and HBM contention of a full batch
// (a unit alone on a few SMs would run from L2 and look faster than it is).
// Two runs (kTuneOuterA and kTuneOuterB outer iterations) give the time per
// outer iteration by difference.  -1 for sizes above `total`.
gadi_status tune_class(gadi_handle *h, const void *k, size_t smem, const std::vector<Params> &cls, int prec,
                       int total, cudaStream_t st, std::vector<double> &t_outer, int nr = 1, int res_optin = 0)
{
    const int nc = (int)(sizeof kTuneSizes / sizeof kTuneSizes[0]);
    t_outer.assign(nc, -1.0);
    DevBuf xs;
    const size_t vb = sizeof(double) * (size_t)h->nelem * nr; // one unit's x (nr right-hand sides)
    CK(cudaMalloc(&xs.p, vb * (size_t)total));
    for (int i = 0; i < nc; i++) {
        const int sz = kTuneSizes[i];
        if (sz > total) continue;
        if (res_optin > 0) {
            // the resident H-solve: sizes whose row share fits
            if (!res_allowed(h->nx, h->ny, sz, res_optin)) continue;
            smem = res_smem(h->nx, h->ny, sz);
        }
        const int ng = total / sz;
        double med[2] = {0.0, 0.0};
        for (int run = 0; run < 2; run++) {
            const int outer = run == 0 ? kTuneOuterA : kTuneOuterB;
            // the copies cycle through the class's units (their alpha values
            // and right-hand sides)
            std::vector<Params> u(ng);
            std::vector<int> ord(ng);
            for (int j = 0; j < ng; j++) {
                u[j] = cls[(size_t)j % cls.size()];
                u[j].x = (double *)xs.p + (size_t)j * h->nelem * nr;
                u[j].tol = 0.0;
                u[j].maxit = outer;
                u[j].outer_win = 0;
                ord[j] = j;
            }
            CK(cudaMemsetAsync(xs.p, 0, vb * (size_t)ng, st));
            BatchLayout lay;
            lay.gsize.assign(ng, sz);
            lay.gclass.assign(ng, 0);
            lay.blocks = ng * sz;
            std::vector<Ctl> c;
            std::vector<unsigned long long> a, b;
            gadi_status s = run_batch(h, k, smem, u, {0, ng}, ord, lay, h->nelem, prec, outer + 2, st, c, a, b,
                                      nullptr, nr);
            if (s != GADI_OK) return s;
            std::vector<double> per(ng);
            for (int j = 0; j < ng; j++) per[j] = (double)(b[j] - a[j]) * 1e-9;
            std::nth_element(per.begin(), per.begin() + ng / 2, per.end());
            med[run] = per[ng / 2];
        }
        // (a unit that converged or stopped early in the trial: its time over
        // the longer run)
        const double d = (med[1] - med[0]) / (kTuneOuterB - kTuneOuterA);
        t_outer[i] = d > 0 ? d : med[1] / kTuneOuterB;
    }
    return GADI_OK;
}

// Groups per class for a given group size per class: in proportion to each
// class's work (units x block-seconds per unit), at least one each, then one
// at a time to the class that would finish last while the grid has room.
// Returns false if the classes' single groups do not fit in the grid.
bool assign_groups(const std::vector<int> &sz, const std::vector<double> &T, const std::vector<int> &count,
                   int total, std::vector<int> &g)
{
    const int ncl = (int)sz.size();
    g.assign(ncl, 1);
    double wsum = 0.0;
    std::vector<double> w(ncl);
    for (int c = 0; c < ncl; c++) wsum += (w[c] = count[c] * sz[c] * T[c]);
    int used = 0;
    for (int c = 0; c < ncl; c++) {
        g[c] = std::max(1, std::min(count[c], (int)std::floor(total * w[c] / wsum / sz[c])));
        used += g[c] * sz[c];
    }
    // over the grid: take groups back from the class with the most blocks
    while (used > total) {
        int pick = -1;
        for (int c = 0; c < ncl; c++)
            if (g[c] > 1 && (pick < 0 || g[c] * sz[c] > g[pick] * sz[pick])) pick = c;
        if (pick < 0) return false;
        g[pick]--;
        used -= sz[pick];
    }
    for (;;) {
        int pick = -1;
        double worst = -1.0;
        for (int c = 0; c < ncl; c++) {
            const double m = std::ceil((double)count[c] / g[c]) * T[c];
            if (g[c] < count[c] && used + sz[c] <= total && m > worst) {
                worst = m;
                pick = c;
            }
        }
        if (pick < 0) break;
        g[pick]++;
        used += sz[pick];
    }
    return true;
}

// Estimated finish time of a layout: the class whose units, taken in rounds
// of its group count, end last (stealing across classes only shortens it).
double finish_estimate(const std::vector<int> &g, const std::vector<double> &T, const std::vector<int> &count)
{
    double m = 0.0;
    for (size_t c = 0; c < g.size(); c++) m = std::max(m, std::ceil((double)count[c] / g[c]) * T[c]);
    return m;
}

// The layout: one size per class and groups per class, every block used.
// Size: fixed, or (tuned) each class starts at the size with the fewest
// block-seconds per unit and moves, one class at a time, to the size that
// lowers the estimated finish time most.  Classes are in size order
// (largest first).
BatchLayout make_layout(const std::vector<long long> &side, const std::vector<int> &count,
                        const std::vector<std::vector<double>> &t_outer, int fixed, int total,
                        std::vector<int> *chosen, double *estimate)
{
    const int ncl = (int)side.size(), nc = (int)(sizeof kTuneSizes / sizeof kTuneSizes[0]);
    std::vector<int> sz(ncl, 1), g;
    std::vector<double> T(ncl, 1.0);
    // a unit's time on a group of kTuneSizes[i] blocks: the class's time per
    // outer iteration times the grid's side (the outer iteration count of HSS
    // near alpha* grows with the side)
    auto unit_time = [&](int c, int i) { return t_outer[c][i] * (double)side[c]; };
    std::vector<int> bi(ncl, -1);
    for (int c = 0; c < ncl; c++) {
        if (fixed > 0) {
            sz[c] = std::min(fixed, total);
            // no timings: work in proportion to points x outer iterations
            T[c] = (double)side[c] * (double)side[c] * (double)side[c] / sz[c];
            continue;
        }
        // start from the size with the fewest block-seconds per unit
        for (int i = 0; i < nc; i++)
            if (t_outer[c][i] > 0 &&
                (bi[c] < 0 || kTuneSizes[i] * t_outer[c][i] <= kTuneSizes[bi[c]] * t_outer[c][bi[c]] * 1.0000001))
                bi[c] = i;
        if (bi[c] < 0) return BatchLayout{};
        sz[c] = kTuneSizes[bi[c]];
        T[c] = unit_time(c, bi[c]);
    }
    bool ok = assign_groups(sz, T, count, total, g);
    double best = ok ? finish_estimate(g, T, count) : HUGE_VAL;
    if (fixed <= 0) {
        // then one class at a time to the size that lowers the estimated
        // finish time most, until no change helps (a class with little work
        // whose cheapest size is large otherwise holds blocks the classes
        // with the work need, and a class of few large units may finish
        // sooner on fewer, larger groups)
        for (int round = 0; round < 8 * ncl + 8; round++) {
            int bc = -1, bsz = -1;
            double bt = 0.0, bval = best;
            for (int c = 0; c < ncl; c++)
                for (int i = 0; i < nc; i++) {
                    if (t_outer[c][i] <= 0 || kTuneSizes[i] == sz[c] || kTuneSizes[i] > total) continue;
                    std::vector<int> s2 = sz, g2;
                    std::vector<double> T2 = T;
                    s2[c] = kTuneSizes[i];
                    T2[c] = unit_time(c, i);
                    if (!assign_groups(s2, T2, count, total, g2)) continue;
                    const double e = finish_estimate(g2, T2, count);
                    if (e < bval * 0.999) {
                        bval = e;
                        bc = c;
                        bsz = kTuneSizes[i];
                        bt = T2[c];
                    }
                }
            if (bc < 0) break;
            sz[bc] = bsz;
            T[bc] = bt;
            best = bval;
            ok = true;
        }
        ok = assign_groups(sz, T, count, total, g);
    }
    if (!ok) return BatchLayout{};
    BatchLayout lay;
    for (int c = 0; c < ncl; c++)
        for (int j = 0; j < g[c]; j++) {
            lay.gsize.push_back(sz[c]);
            lay.gclass.push_back(c);
            lay.blocks += sz[c];
        }
    if (chosen) *chosen = sz;
    if (estimate) *estimate = finish_estimate(g, T, count);
    return lay;
}

} // namespace

extern "C" {

gadi_status gadi_solve_batched(gadi_handle *const *hs, int nsys, int nrhs, const double *const *b,
                               double *const *x, const double *alpha, double omega, gadi_prec u_high,
                               gadi_prec u_low, double tol, int maxit, const gadi_opts *opts,
                               gadi_stats *per_unit)
{
    if (!hs || !b || !x || !alpha || nsys <= 0 || nrhs <= 0) return GADI_ERR_INVALID;
    if (!std::isfinite(omega) || std::isnan(tol)) return GADI_ERR_NONFINITE;
    if (!(omega >= 0 && omega < 2) || u_high != GADI_FP64 || !(tol >= 0) || maxit < 0) return GADI_ERR_INVALID;
    if (u_low != GADI_FP64 && u_low != GADI_FP32 && u_low != GADI_BF16) return GADI_ERR_INVALID;
    gadi_opts o;
    if (opts) o = *opts;
    else gadi_opts_default(&o, u_low);
    gadi_status s = opts_check(o);
    if (s != GADI_OK) return s;
    const int prec = (int)u_low;
    const int vecw = prec == P_FP64 ? 2 : (prec == P_FP32 ? 4 : 8);
    bool vec = true;
    long long max_n = 0;
    for (int i = 0; i < nsys; i++) {
        if (!hs[i] || !b[i] || !x[i]) return GADI_ERR_INVALID;
        if (hs[i]->kind != GADI_STENCIL_2D5) return GADI_ERR_UNSUPPORTED;
        if (!std::isfinite(alpha[i])) return GADI_ERR_NONFINITE;
        if (!(alpha[i] > 0)) return GADI_ERR_INVALID;
        if (!is_device_ptr(b[i]) || !is_device_ptr(x[i])) return GADI_ERR_INVALID;
        if (hs[i]->nx % vecw || !aligned16(b[i]) || !aligned16(x[i]) || (hs[i]->nelem & 1)) vec = false;
        max_n = std::max(max_n, hs[i]->nelem);
    }
    gadi_handle *h0 = hs[0];
    cudaStream_t st = (cudaStream_t)o.stream;
    size_t smem = 0;
    // four right-hand sides of a system interleaved in one unit ([n][4]
    // vectors, FP32 inner solves), or a unit per right-hand side
    const bool inter = nrhs == 4 && prec == P_FP32 && o.u_r == GADI_FP64 && o.batch_interleave != 0;
    const int nr = inter ? 4 : 1;
    // units with the SM-resident H-solve (p in shared memory): FP32 / BF16,
    // 16-byte rows, an FP64 residual, opts->h_resident >= 1
    bool res = !inter && vec && o.h_resident >= 1 && (prec == P_FP32 || prec == P_BF16) && o.u_r == GADI_FP64;
    // the dynamic shared memory a block of the resident kernel may take: the
    // opt-in limit less the kernel's static shared memory
    int optin = 0;
    if (res) {
        CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h0->device));
        cudaFuncAttributes fa;
        CK(cudaFuncGetAttributes(&fa, kernel_batched_2d5_res(prec)));
        optin -= (int)fa.sharedSizeBytes;
        res = optin > 0;
    }
    for (int i = 0; i < nsys && res; i++) {
        // a fixed group size must suit every system; tuned, some candidate
        // size must (else the batch takes the streaming H-solve)
        if (o.batch_group > 0) {
            res = res_allowed(hs[i]->nx, hs[i]->ny, o.batch_group, optin);
        } else {
            bool any = false;
            for (int sz : kTuneSizes)
                any = any || ((o.max_blocks <= 0 || sz <= o.max_blocks) && res_allowed(hs[i]->nx, hs[i]->ny, sz, optin));
            res = any;
        }
    }
    const void *k = inter ? kernel_batched4_2d5(&smem)
                          : (res ? kernel_batched_2d5_res(prec)
                                 : kernel_batched_2d5(prec, vec ? 1 : 0, &smem, o.u_r == GADI_FP64X2));
    if (!k) return GADI_ERR_UNSUPPORTED;
    if (res) smem = (size_t)optin; // the occupancy at the largest share; each launch takes what it needs
    if (smem) CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreadsHost, smem));
    int total = per_sm * h0->nsm;
    if (o.max_blocks > 0) total = std::min(total, o.max_blocks);
    const int nunits = inter ? nsys : nsys * nrhs;
    auto sys_of = [&](int u) { return inter ? u : u / nrhs; };
    // size classes: systems of the same grid, largest first
    std::vector<int> sys_class(nsys, -1);
    std::vector<int> cls_sys; // a representative system per class
    {
        std::vector<int> by_size(nsys);
        for (int i = 0; i < nsys; i++) by_size[i] = i;
        std::stable_sort(by_size.begin(), by_size.end(),
                         [&](int a_, int c_) { return hs[a_]->nelem > hs[c_]->nelem; });
        for (int i : by_size) {
            for (int c = 0; c < (int)cls_sys.size(); c++)
                if (hs[cls_sys[c]]->nx == hs[i]->nx && hs[cls_sys[c]]->ny == hs[i]->ny) sys_class[i] = c;
            if (sys_class[i] < 0) {
                sys_class[i] = (int)cls_sys.size();
                cls_sys.push_back(i);
            }
        }
    }
    const int ncl = (int)cls_sys.size();
    std::vector<Params> units(nunits);
    for (int u = 0; u < nunits; u++) {
        const int sy = sys_of(u), j = inter ? 0 : u % nrhs;
        gadi_handle *h = hs[sy];
        Params &P = units[u];
        fill_base(h, P, prec);
        fill_inner(h, P, prec, alpha[sy], omega);
        P.mode = MODE_SOLVE;
        P.b = b[sy] + (size_t)j * h->nelem;
        P.x = x[sy] + (size_t)j * h->nelem;
        P.tol = tol;
        P.tol_h = o.tol_h;
        P.tol_s = o.tol_s;
        P.maxit = maxit;
        P.maxit_inner = o.maxit_inner;
        P.inner_stag = o.inner_stag;
        P.outer_win = o.outer_stag_window;
        P.ur_dd = o.u_r == GADI_FP64X2;
        P.pointwise = o.s_pointwise;
    }
    // units by class (largest system first), in unit order within a class
    std::vector<int> class_begin(ncl + 1, 0), order;
    std::vector<int> count(ncl, 0);
    std::vector<long long> side(ncl);
    for (int c = 0; c < ncl; c++) {
        for (int u = 0; u < nunits; u++)
            if (sys_class[sys_of(u)] == c) order.push_back(u);
        class_begin[c + 1] = (int)order.size();
        count[c] = class_begin[c + 1] - class_begin[c];
        side[c] = std::max<long long>(hs[cls_sys[c]]->nx, hs[cls_sys[c]]->ny);
    }
    // group sizes: fixed (batch_group > 0) or tuned per class on the device
    // (a few outer iterations of one unit on one group of each size, kept
    // for the process by grid, precision and options)
    std::vector<std::vector<double>> t_outer(ncl);
    if (o.batch_group <= 0) {
        for (int c = 0; c < ncl; c++) {
            gadi_handle *hc = hs[cls_sys[c]];
            std::vector<Params> cls;
            std::vector<double> al;
            for (int q = class_begin[c]; q < class_begin[c + 1]; q++) {
                cls.push_back(units[order[q]]);
                al.push_back(alpha[sys_of(order[q])]);
            }
            std::vector<long long> key = tune_key(hc, prec, o, total, al);
            key.push_back(nr);
            key.push_back(res);
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                auto it = g_tune.find(key);
                if (it != g_tune.end()) t_outer[c] = it->second;
            }
            if (t_outer[c].empty()) {
                if ((s = tune_class(hc, k, smem, cls, prec, total, st, t_outer[c], nr, res ? optin : 0)) != GADI_OK)
                    return s;
                std::lock_guard<std::mutex> lk(g_tune_mu);
                g_tune[key] = t_outer[c];
            }
        }
    }
    std::vector<int> chosen;
    double est = 0.0;
    const BatchLayout lay = make_layout(side, count, t_outer, o.batch_group, total, &chosen, &est);
    if (lay.blocks <= 0) return GADI_ERR_INVALID;
    if (const char *v = std::getenv("GADI_TUNE_VERBOSE"); v && *v == '1') {
        // diagnostic: the tuner's table and the layout taken, on stderr
        for (int c = 0; c < ncl; c++) {
            int groups = 0;
            for (int g : lay.gclass) groups += g == c;
            std::fprintf(stderr, "gadi batch class %d: %lld x %lld, %d units, size %d, %d groups; s/outer:", c,
                         (long long)hs[cls_sys[c]]->nx, (long long)hs[cls_sys[c]]->ny, count[c],
                         chosen.empty() ? 0 : chosen[c], groups);
            for (size_t i = 0; i < t_outer[c].size(); i++) std::fprintf(stderr, " %g", t_outer[c][i]);
            std::fprintf(stderr, "\n");
        }
        std::fprintf(stderr, "gadi batch layout: %d blocks, estimated finish %g s\n", lay.blocks, est);
    }
    // resident units: the group sizes each class admits, and the shared
    // memory of the largest share a group may take (its own class or, by
    // stealing, a smaller one)
    std::vector<int> gmin(ncl, 1), gmax(ncl, 1 << 30);
    if (res) {
        smem = 0;
        for (int c = 0; c < ncl; c++) {
            const gadi_handle *hc = hs[cls_sys[c]];
            gmax[c] = (int)std::min<long long>(hc->ny, 1 << 30);
            gmin[c] = 1 << 30;
            // the share shrinks as the group grows: the smallest size that fits
            for (int sz = 1; sz <= std::min(gmax[c], total) && gmin[c] == (1 << 30); sz++)
                if (res_allowed(hc->nx, hc->ny, sz, optin)) gmin[c] = sz;
        }
        for (size_t g = 0; g < lay.gsize.size(); g++) {
            const int sz = lay.gsize[g], c0 = lay.gclass[g];
            if (sz < gmin[c0] || sz > gmax[c0]) return GADI_ERR_INVALID; // the tuner admits no such size
            for (int c = c0; c < ncl; c++)
                if (sz >= gmin[c] && sz <= gmax[c])
                    smem = std::max(smem, res_smem(hs[cls_sys[c]]->nx, hs[cls_sys[c]]->ny, sz));
        }
    }
    const int hist_len = maxit + 2;
    std::vector<Ctl> hc;
    std::vector<unsigned long long> t0, t1;
    float ms = 0.f;
    if ((s = run_batch(h0, k, smem, units, class_begin, order, lay, max_n, prec, hist_len, st, hc, t0, t1, &ms,
                       nr, &gmin, &gmax)) != GADI_OK)
        return s;
    gadi_status worst = GADI_OK;
    // (system, right-hand side) q = s * nrhs + j: its unit and control block
    for (int q = 0; q < nsys * nrhs; q++) {
        const int u = inter ? q / nrhs : q;
        const Ctl &c = hc[q];
        if (c.status != GADI_OK && worst == GADI_OK) worst = (gadi_status)c.status;
        if (per_unit) {
            gadi_stats &S = per_unit[q];
            S.outer_its = c.outer_its;
            S.inner_its_h = c.inner_h;
            S.inner_its_s = c.inner_s;
            S.relres = c.relres;
            S.r0_norm = c.r0;
            S.seconds = (double)(t1[u] - t0[u]) * 1e-9;
            S.status = c.status;
            S.blocks = c.pad; // the size of the group that ran the unit
            S.alpha = alpha[q / nrhs];
            S.restarts = 0;
            S.h_resident = res ? 1 : 0;
            S.s_resident = 0;
            S.backward_err = -1.0;
        }
    }
    return worst;
}

gadi_status gadi_batch_plan(int ncl, const long long *side, const int *count, const double *t_outer, int fixed,
                            int total, int *size, int *groups, double *estimate)
{
    constexpr int nc = (int)(sizeof kTuneSizes / sizeof kTuneSizes[0]);
    if (ncl <= 0 || !side || !count || !size || !groups || total <= 0 || (fixed <= 0 && !t_outer))
        return GADI_ERR_INVALID;
    std::vector<long long> sd(side, side + ncl);
    std::vector<int> cn(count, count + ncl);
    std::vector<std::vector<double>> t(ncl, std::vector<double>(nc, -1.0));
    for (int c = 0; c < ncl; c++) {
        if (sd[c] <= 0 || cn[c] <= 0) return GADI_ERR_INVALID;
        if (t_outer)
            for (int i = 0; i < nc; i++) t[c][i] = t_outer[(size_t)c * nc + i];
    }
    std::vector<int> chosen;
    double est = 0.0;
    const BatchLayout lay = make_layout(sd, cn, t, fixed, total, &chosen, &est);
    if (lay.blocks <= 0) return GADI_ERR_INVALID;
    for (int c = 0; c < ncl; c++) {
        size[c] = chosen[c];
        groups[c] = 0;
    }
    for (int g : lay.gclass) groups[g]++;
    if (estimate) *estimate = est;
    return GADI_OK;
}

gadi_status gadi_apply(gadi_handle *h, gadi_op op, const double *x, double *y, void *stream)
{
    if (!h || !x || !y || op < GADI_OP_A || op > GADI_OP_AT || x == y) return GADI_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t vb = sizeof(double) * (size_t)h->nelem;
    const bool xd = is_device_ptr(x), yd = is_device_ptr(y);
    if (!xd || !yd)
        if (!h->d_stage) CK(cudaMalloc(&h->d_stage, 2 * vb));
    const double *dx = xd ? x : h->d_stage;
    double *dy = yd ? y : h->d_stage + h->nelem;
    if (!xd) CK(cudaMemcpyAsync((void *)dx, x, vb, cudaMemcpyHostToDevice, st));
    gadi_status s = apply_dev(h, op, dx, dy, st);
    if (s != GADI_OK) return s;
    if (!yd) {
        CK(cudaMemcpyAsync(y, dy, vb, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return GADI_OK;
}

gadi_status gadi_norm2_estimate(gadi_handle *h, int iters, double *out, void *stream)
{
    if (!h || !out || iters <= 0) return GADI_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    const long long m = h->nelem;
    if (!h->d_pw) CK(cudaMalloc(&h->d_pw, sizeof(double) * (3 * (size_t)m + 2)));
    double *v = h->d_pw, *t = v + m, *wv = t + m, *acc = wv + m;
    const int gb = std::max(1, h->nsm * 4);
    k_init_pw<<<gb, 256, 0, st>>>(v, m);
    CK(cudaGetLastError());
    double hs = 0.0;
    for (int it = 0; it < iters + 1; it++) {
        // v <- v / ||v||
        CK(cudaMemsetAsync(acc, 0, sizeof(double), st));
        k_dot<<<gb, 256, 0, st>>>(v, v, m, acc);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&hs, acc, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (!(hs > 0)) {
            *out = 0.0;
            return GADI_OK;
        }
        if (it == iters) break;
        k_scale_copy<<<gb, 256, 0, st>>>(v, 1.0 / std::sqrt(hs), m, v);
        gadi_status s = apply_dev(h, GADI_OP_A, v, t, st);
        if (s != GADI_OK) return s;
        if ((s = apply_dev(h, GADI_OP_AT, t, wv, st)) != GADI_OK) return s;
        std::swap(v, wv);
    }
    // after the loop ||v|| = ||A^T A v_prev|| with ||v_prev|| = 1
    *out = std::sqrt(std::sqrt(hs));
    return GADI_OK;
}

gadi_status gadi_step_residual(gadi_handle *h, gadi_prec u_low, const double *b, const double *x,
                               const void *y, double *x_out, double *r_out, void *rs, double *rnorm,
                               void *stream)
{
    return gadi_step_residual_ur(h, GADI_FP64, u_low, b, x, y, x_out, r_out, nullptr, rs, rnorm, stream);
}

gadi_status gadi_step_residual_ur(gadi_handle *h, gadi_prec u_r, gadi_prec u_low, const double *b,
                                  const double *x, const void *y, double *x_out, double *r_out,
                                  double *r_lo_out, void *rs, double *rnorm, void *stream)
{
    if (!h || !b || !x || !x_out || !rs || x_out == x) return GADI_ERR_INVALID;
    if (u_low != GADI_FP64 && u_low != GADI_FP32 && u_low != GADI_BF16) return GADI_ERR_INVALID;
    if (u_r != GADI_FP64 && u_r != GADI_FP64X2) return GADI_ERR_INVALID;
    const int prec = (int)u_low;
    cudaStream_t st = (cudaStream_t)stream;
    Work w;
    gadi_status s = ensure_ws(h, prec, &w);
    if (s != GADI_OK) return s;
    Params P;
    fill_base(h, P, prec);
    P.mode = MODE_RESIDUAL;
    set_work(P, w);
    P.b = b;
    P.x = (double *)x;
    P.y = (void *)y;
    P.x1 = x_out;
    P.r_out = r_out;
    P.r_lo_out = r_lo_out;
    P.ur_dd = u_r == GADI_FP64X2;
    // an FP64 residual has no low part
    if (r_lo_out && !P.ur_dd) CK(cudaMemsetAsync(r_lo_out, 0, sizeof(double) * (size_t)h->nelem, st));
    P.r = rs;
    P.maxit = 1;
    if ((s = launch(h, prec, P, 0, st, nullptr)) != GADI_OK) return s;
    if ((s = finish(h, st)) != GADI_OK) return s;
    if (rnorm) *rnorm = h->h_ctl->rnorm;
    return GADI_OK;
}

gadi_status gadi_step_solve_h(gadi_handle *h, double alpha, gadi_prec u_low, const void *rs, void *z,
                              double tol, int maxit, int stag, int *its, void *stream)
{
    if (!h || !rs || !z || !(alpha > 0) || !(tol >= 0) || maxit < 0 || stag < 0) return GADI_ERR_INVALID;
    if (u_low != GADI_FP64 && u_low != GADI_FP32 && u_low != GADI_BF16) return GADI_ERR_INVALID;
    const int prec = (int)u_low;
    cudaStream_t st = (cudaStream_t)stream;
    Work w;
    gadi_status s = ensure_ws(h, prec, &w);
    if (s != GADI_OK) return s;
    if (h->kind == GADI_CSR && (s = ensure_csr_ops(h, prec, alpha)) != GADI_OK) return s;
    CK(cudaMemcpyAsync(w.r, rs, elem_bytes(prec) * (size_t)h->nelem, cudaMemcpyDeviceToDevice, st));
    Params P;
    fill_base(h, P, prec);
    fill_inner(h, P, prec, alpha, 1.0);
    P.mode = MODE_SOLVE_H;
    set_work(P, w);
    P.z = z;
    P.tol_h = tol;
    P.maxit_inner = maxit;
    P.inner_stag = stag;
    P.maxit = 1;
    P.resident = prec == P_BF16 ? 1 : 2; // as gadi_opts_default
    if ((s = launch(h, prec, P, 0, st, nullptr)) != GADI_OK) return s;
    if ((s = finish(h, st)) != GADI_OK) return s;
    if (its) *its = (int)h->h_ctl->inner_h;
    return GADI_OK;
}

gadi_status gadi_step_solve_s(gadi_handle *h, double alpha, double omega, gadi_prec u_low, const void *z,
                              void *y, double tol, int maxit, int stag, int pointwise, int *its,
                              void *stream)
{
    if (!h || !z || !y || !(alpha > 0) || !(omega >= 0 && omega < 2) || !(tol >= 0) || maxit < 0 || stag < 0)
        return GADI_ERR_INVALID;
    if (u_low != GADI_FP64 && u_low != GADI_FP32 && u_low != GADI_BF16) return GADI_ERR_INVALID;
    const int prec = (int)u_low;
    cudaStream_t st = (cudaStream_t)stream;
    Work w;
    gadi_status s = ensure_ws(h, prec, &w);
    if (s != GADI_OK) return s;
    if (h->kind == GADI_CSR && (s = ensure_csr_ops(h, prec, alpha)) != GADI_OK) return s;
    Params P;
    fill_base(h, P, prec);
    fill_inner(h, P, prec, alpha, omega);
    P.mode = MODE_SOLVE_S;
    set_work(P, w);
    P.z = (void *)z;
    P.y = y;
    P.tol_s = tol;
    P.maxit_inner = maxit;
    P.inner_stag = stag;
    P.pointwise = pointwise;
    P.maxit = 1;
    if ((s = launch(h, prec, P, 0, st, nullptr)) != GADI_OK) return s;
    if ((s = finish(h, st)) != GADI_OK) return s;
    if (its) *its = (int)h->h_ctl->inner_s;
    return GADI_OK;
}

} // extern "C"
