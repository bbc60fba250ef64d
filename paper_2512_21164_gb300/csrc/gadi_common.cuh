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
// The same rounding by the conversion instruction (cvt.rn.bf16.f32: round to
// nearest even, subnormals kept): one instruction instead of the integer
// sequence above, which the inner solves' stores otherwise spend most of
// their integer-pipe issue slots on.  Equal to f32_to_bf16 for every
// non-NaN input (NaN gives some quiet NaN).
__device__ __forceinline__ uint16_t f32_to_bf16_cvt(float f)
{
    unsigned short h;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(f));
    return (uint16_t)h;
}

// two floats rounded to BF16 (nearest even) by one instruction and returned
// as floats: `hi` from the upper half of the packed pair, `lo` the lower.  The
// same rounding as f32_to_bf16_cvt for each value.
__device__ __forceinline__ void f32x2_round_bf16(float a, float b, float &ra, float &rb)
{
    unsigned d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(a), "f"(b));
    ra = __uint_as_float(d & 0xffff0000u);
    rb = __uint_as_float(d << 16);
}

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
// binary32/BF16 <-> binary64 conversions on the integer pipe.  On GB300 the
// hardware conversions between FP32 and FP64 issue on the FP64 pipe, at about
// 2 per clock per SM (the same rate as an FP64 fused multiply-add, against
// some 64 integer operations), and the FP64 residual of each outer iteration
// is bound by that pipe.  The common cases -- zero and results in the normal
// binary32 range -- are therefore assembled from the IEEE 754 fields
// (sign, biased exponent, significand) with integer operations; subnormal,
// infinite, NaN and out-of-range cases fall back to the hardware conversion.
// The results equal the hardware conversions bit for bit (checked on the
// device by gadi_selftest_convert).
// ---------------------------------------------------------------------------
// exact widening: rebias the exponent (1023 - 127 = 896), shift the
// 23-bit significand into the top of the 52-bit one
__device__ __forceinline__ double f32_to_f64_fast(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu;
    if (e - 1u < 254u) {
        const uint32_t hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
        return __hiloint2double((int)hi, (int)(u << 29));
    }
    if ((u & 0x7fffffffu) == 0u) return __hiloint2double((int)u, 0);
    return (double)f;
}
// round to nearest, ties to even, keeping `keep` of the 52 significand bits:
// the top `keep` bits with the exponent above them, plus one if the discarded
// part exceeds half an ulp or equals it with an odd kept part (a carry out of
// the significand moves into the exponent, and past the largest finite
// exponent gives infinity, as rounding requires)
// `beyond` breaks an exact tie for a value that is the double plus a small
// remainder of the sign it gives: +1 (the value lies past the cut: round
// up), -1 (short of it: round down), 0 (no remainder: ties to even).
template <int KEEP>
__device__ __forceinline__ uint32_t f64_round_fields(uint64_t u, uint32_t e32, int beyond = 0)
{
    constexpr int DROP = 52 - KEEP;
    const uint64_t mant = u & 0xfffffffffffffull;
    uint32_t bits = (e32 << KEEP) | (uint32_t)(mant >> DROP);
    const uint64_t rem = mant & ((1ull << DROP) - 1ull), half = 1ull << (DROP - 1);
    const bool up = rem > half || (rem == half && (beyond > 0 || (beyond == 0 && (bits & 1u))));
    bits += up ? 1u : 0u;
    return bits;
}
__device__ __forceinline__ float f64_to_f32_fast(double d)
{
    const uint64_t u = (uint64_t)__double_as_longlong(d);
    const uint32_t ed = (uint32_t)(u >> 52) & 0x7ffu, sign = (uint32_t)(u >> 32) & 0x80000000u;
    if (ed - 897u < 254u) return __uint_as_float(sign | f64_round_fields<23>(u, ed - 896u));
    if ((u << 1) == 0ull) return __uint_as_float(sign);
    return __double2float_rn(d);
}
__device__ __forceinline__ uint16_t f64_to_bf16_fast(double d)
{
    const uint64_t u = (uint64_t)__double_as_longlong(d);
    const uint32_t ed = (uint32_t)(u >> 52) & 0x7ffu, sign = (uint32_t)(u >> 48) & 0x8000u;
    if (ed - 897u < 254u) return (uint16_t)(sign | f64_round_fields<7>(u, ed - 896u));
    if ((u << 1) == 0ull) return (uint16_t)sign;
    return f64_to_bf16(d);
}

// the unevaluated pair hi + lo (|lo| <= ulp(hi)/2) rounded to binary32 /
// BF16: hi's rounding, except that an exact tie of hi is decided by lo's
// sign; outside the normal binary32 range hi alone is rounded
__device__ __forceinline__ int f64x2_beyond(double hi, double lo)
{
    return lo == 0.0 ? 0 : ((lo > 0.0) == (hi > 0.0) ? 1 : -1);
}
__device__ __forceinline__ float f64x2_to_f32(double hi, double lo)
{
    const uint64_t u = (uint64_t)__double_as_longlong(hi);
    const uint32_t ed = (uint32_t)(u >> 52) & 0x7ffu, sign = (uint32_t)(u >> 32) & 0x80000000u;
    if (ed - 897u < 254u) return __uint_as_float(sign | f64_round_fields<23>(u, ed - 896u, f64x2_beyond(hi, lo)));
    return f64_to_f32_fast(hi);
}
__device__ __forceinline__ uint16_t f64x2_to_bf16(double hi, double lo)
{
    const uint64_t u = (uint64_t)__double_as_longlong(hi);
    const uint32_t ed = (uint32_t)(u >> 52) & 0x7ffu, sign = (uint32_t)(u >> 48) & 0x8000u;
    if (ed - 897u < 254u) return (uint16_t)(sign | f64_round_fields<7>(u, ed - 896u, f64x2_beyond(hi, lo)));
    return f64_to_bf16_fast(hi);
}

// error-free transformations in FP64: a + b = s + e exactly (Knuth's
// TwoSum, no ordering condition), a * b = p + e exactly (fused
// multiply-add), both as in Ogita, Rump & Oishi 2005
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e)
{
    s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(double a, double b, double &p, double &e)
{
    p = __dmul_rn(a, b);
    e = fma(a, b, -p);
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
    __device__ static S from_f64x2(double hi, double) { return hi; }
    __device__ static double to_f64(S s) { return s; }
};
template <> struct Prec<P_FP32> {
    using S = float; using C = float; static constexpr int VEC = 4;
    __device__ static C ld(S s) { return s; }
    __device__ static S st(C c) { return c; }
    __device__ static S from_f64(double d) { return f64_to_f32_fast(d); }
    __device__ static S from_f64x2(double hi, double lo) { return f64x2_to_f32(hi, lo); }
    __device__ static double to_f64(S s) { return f32_to_f64_fast(s); }
};
template <> struct Prec<P_BF16> {
    using S = uint16_t; using C = float; static constexpr int VEC = 8;
    __device__ static C ld(S s) { return bf16_to_f32(s); }
    __device__ static S st(C c) { return f32_to_bf16_cvt(c); }
    __device__ static S from_f64(double d) { return f64_to_bf16_fast(d); }
    __device__ static S from_f64x2(double hi, double lo) { return f64x2_to_bf16(hi, lo); }
    __device__ static double to_f64(S s) { return f32_to_f64_fast(bf16_to_f32(s)); }
};

// ---------------------------------------------------------------------------
// vector loads / stores of W consecutive elements (W * sizeof(T) in
// {2,4,8,16,32,64} bytes; the address must be aligned to min(16, that size))
// ---------------------------------------------------------------------------
// Loads come in two cache policies: `load` (ld.global.cg, L2 only) for data a
// block touches once per phase, and `load_ca` (ld.global.ca, L1 and L2) for
// stencil inputs whose rows neighbouring warps of the same block also read.
// Every buffer read with load_ca is read-only during the phase that reads it;
// the grid barrier between phases (acquire at gpu scope) orders it after the
// writes of the previous phase.
template <class T, int W> struct VecIO {
    static constexpr int BYTES = W * (int)sizeof(T);
    template <bool CA>
    __device__ static void load_p(const T *p, T (&v)[W])
    {
        if constexpr (BYTES >= 16) {
#pragma unroll
            for (int i = 0; i < BYTES / 16; i++) {
                const uint4 *a = reinterpret_cast<const uint4 *>(p) + i;
                reinterpret_cast<uint4 *>(v)[i] = CA ? __ldca(a) : __ldcg(a);
            }
        } else if constexpr (BYTES == 8) {
            const uint2 *a = reinterpret_cast<const uint2 *>(p);
            reinterpret_cast<uint2 *>(v)[0] = CA ? __ldca(a) : __ldcg(a);
        } else if constexpr (BYTES == 4) {
            const unsigned *a = reinterpret_cast<const unsigned *>(p);
            reinterpret_cast<unsigned *>(v)[0] = CA ? __ldca(a) : __ldcg(a);
        } else {
            const unsigned short *a = reinterpret_cast<const unsigned short *>(p);
            reinterpret_cast<unsigned short *>(v)[0] = CA ? __ldca(a) : __ldcg(a);
        }
    }
    __device__ static void load(const T *p, T (&v)[W]) { load_p<false>(p, v); }
    __device__ static void load_ca(const T *p, T (&v)[W]) { load_p<true>(p, v); }
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
// the blocks working on one system: the whole grid for a single solve, a
// group of blocks for one system of a batch
// ---------------------------------------------------------------------------
struct VGrid {
    int b; // this block's index in the group
    int n; // blocks in the group
    __device__ long long tid() const { return (long long)b * blockDim.x + threadIdx.x; }
    __device__ long long nthreads() const { return (long long)n * blockDim.x; }
    __device__ long long warp() const { return (long long)b * (blockDim.x >> 5) + (threadIdx.x >> 5); }
    __device__ long long nwarps() const { return (long long)n * (blockDim.x >> 5); }
};
__device__ __forceinline__ VGrid whole_grid() { return VGrid{(int)blockIdx.x, (int)gridDim.x}; }

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

__device__ __forceinline__ unsigned long long atom_add_acq_rel_u64(unsigned long long *p, unsigned long long v)
{
    unsigned long long old;
    asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long atom_add_release_u64(unsigned long long *p, unsigned long long v)
{
    unsigned long long old;
    asm volatile("atom.add.release.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

struct GridSync {
    unsigned long long *counter; // zeroed before launch
    int *abort_flag;             // zeroed before launch; 1 = a wait timed out
    unsigned nblocks;
    unsigned long long timeout_ns = kBarrierTimeoutNs;

    // Arrival is one acquire-release add per block (after a block barrier,
    // so it publishes the whole block's writes); the block whose add
    // completes the count goes on at once, the others poll with acquire
    // loads.  Returns false if this block must unwind (timeout here or
    // elsewhere).
    __device__ bool sync() const
    {
        __shared__ int s_ok;
        __syncthreads();
        if (threadIdx.x == 0) {
            int ok = 1;
            const unsigned long long arrived = atom_add_acq_rel_u64(counter, 1ull) + 1ull;
            // the count this barrier completes at: arrived rounded up to a
            // multiple of nblocks (32-bit division while the count fits)
            const unsigned long long target =
                (arrived >> 32) == 0ull
                    ? (unsigned long long)((((unsigned)arrived + nblocks - 1u) / nblocks) * nblocks)
                    : ((arrived + nblocks - 1ull) / nblocks) * nblocks;
            if (arrived < target) {
                const unsigned long long t0 = globaltimer_ns();
                unsigned spins = 0;
                while (ld_acquire_u64(counter) < target) {
                    if (ld_volatile_int(abort_flag)) { ok = 0; break; }
                    if ((++spins & 63u) == 0 && globaltimer_ns() - t0 > timeout_ns) {
                        atomicExch(abort_flag, 1);
                        ok = 0;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            s_ok = ok;
        }
        __syncthreads();
        return s_ok != 0;
    }

    // sync() in two halves.  arrive() publishes the block's writes (release
    // add; thread 0's value is the count after its add); wait(arrived)
    // returns once every block has arrived.  Between them the block may
    // only read data no other block wrote since the previous barrier.
    __device__ unsigned long long arrive() const
    {
        __syncthreads();
        unsigned long long arrived = 0ull;
        if (threadIdx.x == 0) arrived = atom_add_release_u64(counter, 1ull) + 1ull;
        return arrived;
    }
    __device__ bool wait(unsigned long long arrived) const
    {
        __shared__ int s_ok;
        if (threadIdx.x == 0) {
            int ok = 1;
            const unsigned long long target =
                (arrived >> 32) == 0ull
                    ? (unsigned long long)((((unsigned)arrived + nblocks - 1u) / nblocks) * nblocks)
                    : ((arrived + nblocks - 1ull) / nblocks) * nblocks;
            // at least one acquire load, also when this block arrived last
            const unsigned long long t0 = globaltimer_ns();
            unsigned spins = 0;
            while (ld_acquire_u64(counter) < target) {
                if (ld_volatile_int(abort_flag)) { ok = 0; break; }
                if ((++spins & 63u) == 0 && globaltimer_ns() - t0 > timeout_ns) {
                    atomicExch(abort_flag, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
            s_ok = ok;
        }
        __syncthreads();
        return s_ok != 0;
    }
};

// ---------------------------------------------------------------------------
// tensor memory (TMEM) as per-thread storage
// ---------------------------------------------------------------------------
// TMEM is the 128-lane x 512-column (32-bit) on-chip memory of a Blackwell SM
// that tcgen05 tensor-core instructions accumulate into.  The H-solve uses
// it only as storage: thread i of warp w keeps its values in lane
// 32 (w % 4) + i (a warp may reach only its lane quarter) and in a column
// range of its own.  The 32x32b shape moves one 32-bit word per lane and
// column; x4: four consecutive columns, i.e. 16 bytes per thread.  All of
// these are warp-collective (.sync.aligned): every lane of the warp executes
// them with the same address.  Loads complete at tcgen05.wait::ld, stores at
// tcgen05.wait::st.
__device__ __forceinline__ void tmem_alloc(unsigned *smem_dst, unsigned ncols)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(a), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld4(unsigned taddr, unsigned (&v)[4])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tmem_st4(unsigned taddr, const unsigned (&v)[4])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(v[0]), "r"(v[1]),
                 "r"(v[2]), "r"(v[3])
                 : "memory");
}
// wait for this thread's outstanding TMEM loads; the registers they fill
// pass through the statement so that no use is scheduled before it
template <int N>
__device__ __forceinline__ void tmem_wait_ld(unsigned (&v)[N][4])
{
    static_assert(N == 2 || N == 4, "tmem_wait_ld: 2 or 4 groups");
    if constexpr (N == 2) {
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(v[0][0]), "+r"(v[0][1]), "+r"(v[0][2]), "+r"(v[0][3]), "+r"(v[1][0]), "+r"(v[1][1]),
                       "+r"(v[1][2]), "+r"(v[1][3])::"memory");
    } else {
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(v[0][0]), "+r"(v[0][1]), "+r"(v[0][2]), "+r"(v[0][3]), "+r"(v[1][0]), "+r"(v[1][1]),
                       "+r"(v[1][2]), "+r"(v[1][3]), "+r"(v[2][0]), "+r"(v[2][1]), "+r"(v[2][2]), "+r"(v[2][3]),
                       "+r"(v[3][0]), "+r"(v[3][1]), "+r"(v[3][2]), "+r"(v[3][3])::"memory");
    }
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------------------
// deterministic reductions
// ---------------------------------------------------------------------------
// Each block reduces NV per-thread partial sums (type RT) in a fixed tree and
// writes them to part[k * G + bi] (bi = the block's index among the G blocks
// that work on one system).  After a grid barrier every block
// reads all G partials and sums them in the same fixed order, so every block
// holds bitwise identical totals and takes identical control decisions.
// RT is float for the FP32/BF16 inner solves (FP64 throughput on this GPU is
// about 1/60 of FP32, so double arithmetic on every thread would dominate a
// reduction) and double for FP64 sums (the outer residual norm, GADI-FP64).
template <int NV, class RT>
__device__ __forceinline__ void block_partials_write(const RT (&v)[NV], RT *part, int G, int bi)
{
    __shared__ RT red[NV][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        RT s = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[k][warp] = s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) {
            RT s = lane < nw ? red[k][lane] : RT(0);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) __stcg(part + (size_t)k * G + bi, s);
        }
    }
}

template <int NV, class RT>
__device__ __forceinline__ void grid_partials_sum(const RT *part, int G, RT (&out)[NV])
{
    // One warp issues the loads of all NV x G partials before it adds any of
    // them (one L2 round trip for G <= 32 U: one or two blocks per SM of a
    // 152-SM GPU), sums them in a fixed order and broadcasts through shared
    // memory.
    __shared__ RT res[NV];
    constexpr int U = GADI_THREADS >= 512 ? 5 : 10;
    if ((threadIdx.x >> 5) == 0) {
        const int lane = threadIdx.x & 31;
        RT s[NV];
#pragma unroll
        for (int k = 0; k < NV; k++) s[k] = RT(0);
        for (int base = lane; base < G; base += 32 * U) {
            RT t[NV][U];
#pragma unroll
            for (int k = 0; k < NV; k++)
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int i = base + 32 * u;
                    t[k][u] = i < G ? __ldcg(part + (size_t)k * G + i) : RT(0);
                }
#pragma unroll
            for (int k = 0; k < NV; k++)
#pragma unroll
                for (int u = 0; u < U; u++) s[k] += t[k][u];
        }
#pragma unroll
        for (int k = 0; k < NV; k++) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
            if (lane == 0) res[k] = s[k];
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; k++) out[k] = res[k];
    __syncthreads();
}

} // namespace gadi
