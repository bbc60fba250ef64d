// Shared device-side building blocks of the GADI kernels (sm_103a):
// precision traits, BF16 conversions, 16-byte vector loads/stores, the
// bounded grid barrier of the persistent cooperative kernel and the
// deterministic block/grid reductions.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "gadi_params.h"

namespace gadi {


// status codes (same values as gadi_status)
enum : int {
    ST_OK = 0, ST_NOT_CONVERGED = 1, ST_STAGNATED = 2, ST_DIVERGED = 3,
    ST_ERR_TIMEOUT = -5
};

// ---------------------------------------------------------------------------
// BF16 conversions (round to nearest, ties to even)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint16_t f32_to_bf16(float f)
{
    uint32_t u = __float_as_uint(f);
    if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u); // quiet NaN
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
__device__ __forceinline__ float bf16_to_f32(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// double -> BF16 without double rounding: round to odd at binary32 (truncate,
// then set the last bit if anything was discarded), then round to nearest
// even at BF16.  Binary32 carries 16 more significand bits than BF16, so the
// two-step result equals direct rounding (Boldo & Melquiond, "Emulation of
// FMA and correctly rounded sums: proved algorithms using rounding to odd",
// IEEE TC 2008).
__device__ __forceinline__ uint16_t f64_to_bf16(double d)
{
    float t = __double2float_rz(d);
    if ((double)t != d && !isnan(d)) t = __uint_as_float(__float_as_uint(t) | 1u);
    return f32_to_bf16(t);
}

// ---------------------------------------------------------------------------
// precision traits: storage type S, compute type C, elements per 16 bytes
// ---------------------------------------------------------------------------
template <int P> struct Prec;
template <> struct Prec<P_FP64> {
    using S = double; using C = double; static constexpr int VEC = 2;
    __device__ static C ld(S s) { return s; }
    __device__ static S st(C c) { return c; }
    __device__ static S from_f64(double d) { return d; }
    __device__ static double to_f64(S s) { return s; }
};
template <> struct Prec<P_FP32> {
    using S = float; using C = float; static constexpr int VEC = 4;
    __device__ static C ld(S s) { return s; }
    __device__ static S st(C c) { return c; }
    __device__ static S from_f64(double d) { return __double2float_rn(d); }
    __device__ static double to_f64(S s) { return (double)s; }
};
template <> struct Prec<P_BF16> {
    using S = uint16_t; using C = float; static constexpr int VEC = 8;
    __device__ static C ld(S s) { return bf16_to_f32(s); }
    __device__ static S st(C c) { return f32_to_bf16(c); }
    __device__ static S from_f64(double d) { return f64_to_bf16(d); }
    __device__ static double to_f64(S s) { return (double)bf16_to_f32(s); }
};

// ---------------------------------------------------------------------------
// vector loads / stores of W consecutive elements (W * sizeof(T) in
// {2,4,8,16,32,64} bytes; the address must be aligned to min(16, that size))
// ---------------------------------------------------------------------------
template <class T, int W> struct VecIO {
    static constexpr int BYTES = W * (int)sizeof(T);
    __device__ static void load(const T *p, T (&v)[W])
    {
        if constexpr (BYTES >= 16) {
#pragma unroll
            for (int i = 0; i < BYTES / 16; i++) {
                uint4 q = __ldcg(reinterpret_cast<const uint4 *>(p) + i);
                reinterpret_cast<uint4 *>(v)[i] = q;
            }
        } else if constexpr (BYTES == 8) {
            uint2 q = __ldcg(reinterpret_cast<const uint2 *>(p));
            reinterpret_cast<uint2 *>(v)[0] = q;
        } else if constexpr (BYTES == 4) {
            unsigned q = __ldcg(reinterpret_cast<const unsigned *>(p));
            reinterpret_cast<unsigned *>(v)[0] = q;
        } else {
            unsigned short q = __ldcg(reinterpret_cast<const unsigned short *>(p));
            reinterpret_cast<unsigned short *>(v)[0] = q;
        }
    }
    __device__ static void store(T *p, const T (&v)[W])
    {
        if constexpr (BYTES >= 16) {
#pragma unroll
            for (int i = 0; i < BYTES / 16; i++)
                __stcg(reinterpret_cast<uint4 *>(p) + i, reinterpret_cast<const uint4 *>(v)[i]);
        } else if constexpr (BYTES == 8) {
            __stcg(reinterpret_cast<uint2 *>(p), reinterpret_cast<const uint2 *>(v)[0]);
        } else if constexpr (BYTES == 4) {
            __stcg(reinterpret_cast<unsigned *>(p), reinterpret_cast<const unsigned *>(v)[0]);
        } else {
            __stcg(reinterpret_cast<unsigned short *>(p),
                   reinterpret_cast<const unsigned short *>(v)[0]);
        }
    }
};

// ---------------------------------------------------------------------------
// bounded grid barrier for the persistent cooperative kernel
// ---------------------------------------------------------------------------
// The launch is cooperative (all blocks co-resident), so the barrier always
// completes in a correct program.  Every wait still has a limit: after
// kBarrierTimeoutNs of waiting a block raises the abort flag and returns
// false; blocks that see the flag stop waiting too, and the kernel unwinds.
constexpr unsigned long long kBarrierTimeoutNs = 4000000000ull; // 4 s

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile_int(const int *p)
{
    return *reinterpret_cast<const volatile int *>(p);
}

struct GridSync {
    unsigned long long *counter; // zeroed before launch
    int *abort_flag;             // zeroed before launch; 1 = a wait timed out
    unsigned nblocks;

    // returns false if this block must unwind (timeout here or elsewhere)
    __device__ bool sync() const
    {
        __shared__ int s_ok;
        __syncthreads();
        if (threadIdx.x == 0) {
            int ok = 1;
            __threadfence();
            unsigned long long arrived = atomicAdd(counter, 1ull) + 1ull;
            unsigned long long target = ((arrived + nblocks - 1) / nblocks) * nblocks;
            if (ld_acquire_u64(counter) < target) {
                unsigned long long t0 = globaltimer_ns();
                unsigned spins = 0;
                while (ld_acquire_u64(counter) < target) {
                    if (ld_volatile_int(abort_flag)) { ok = 0; break; }
                    if ((++spins & 63u) == 0 && globaltimer_ns() - t0 > kBarrierTimeoutNs) {
                        atomicExch(abort_flag, 1);
                        ok = 0;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            __threadfence();
            s_ok = ok;
        }
        __syncthreads();
        return s_ok != 0;
    }
};

// ---------------------------------------------------------------------------
// deterministic reductions
// ---------------------------------------------------------------------------
// Each block reduces NV per-thread partial sums (double) in a fixed tree and
// writes them to part[k * G + blockIdx.x].  After a grid barrier every block
// reads all G partials and sums them in the same fixed order, so every block
// holds bitwise identical totals and takes identical control decisions.
template <int NV>
__device__ __forceinline__ void block_partials_write(double (&v)[NV], double *part, int G)
{
    __shared__ double red[NV][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double s = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[k][warp] = s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) {
            double s = lane < nw ? red[k][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) __stcg(part + (size_t)k * G + blockIdx.x, s);
        }
    }
    __syncthreads();
}

template <int NV>
__device__ __forceinline__ void grid_partials_sum(const double *part, int G, double (&out)[NV])
{
    __shared__ double red[NV][32];
    __shared__ double res[NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double s = 0.0;
        for (int i = threadIdx.x; i < G; i += blockDim.x) s += __ldcg(part + (size_t)k * G + i);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[k][warp] = s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) {
            double s = lane < nw ? red[k][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) res[k] = s;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; k++) out[k] = res[k];
    __syncthreads();
}

} // namespace gadi
