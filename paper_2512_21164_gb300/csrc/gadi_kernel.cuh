// The persistent GADI kernel: Algorithm 1 of arXiv 2512.21164 run entirely on
// the device by one cooperative launch.  Every step of an outer iteration is
// a grid-wide "phase"; phases are separated by the bounded grid barrier and
// the scalars of CG / CGNR come from deterministic grid reductions, so every
// block takes the same control decisions without a host round trip.
//
// Phases of one outer iteration (stencil classes):
//   R   x_out = x + y, r = b - A x_out (FP64), r_s = fl_s(r),   sums ||r||^2, ||r_s||^2
//   H1  p = fl_s(r + beta p_old) (halo recomputed), q = H p,      sum p.q
//   H2  z = fl_s(z + a p), r = fl_s(r - a H p) (H p recomputed),  sum r.r
//   S0  g = fl_s(gamma z) (on the fly), t = fl_s(S^T g),           sum t.t
//   S1  p = fl_s(t + beta p_old), u = fl_s(S p),                   sum u.u
//   S2  y = fl_s(y + a p), t = fl_s(t - a S^T u),                  sum t.t
//   SP  (complex class, diagonal S) y = fl_s(g / (alpha + i sigma))
// Matrix-vector products consumed in registers (H p, S^T u) stay in the
// compute type; every vector written to memory is rounded to u_s.
#pragma once
#include "gadi_common.cuh"
#include "gadi_params.h"

namespace gadi {

constexpr int kThreads = GADI_THREADS;
// the SM-resident H-solve phases (instantiated only in their own kernel)
#ifndef GADI_RES_FN
#define GADI_RES_FN __forceinline__
#endif
// resident blocks per SM the register budget is sized for (kThreads each)
#ifndef GADI_MIN_BLOCKS
#define GADI_MIN_BLOCKS (GADI_THREADS >= 512 ? 1 : 512 / GADI_THREADS)
#endif
// 1: 2D inner phases stage rows through shared memory (march_smem)
#ifndef GADI_SMEM_SWEEP
#define GADI_SMEM_SWEEP 0
#endif
// 1: 3D inner phases stage planes of a tile through shared memory
// (march3_smem); 0: the register-ring march
#ifndef GADI_SMEM3
#define GADI_SMEM3 1
#endif


// ---------------------------------------------------------------------------
// arithmetic policies
// ---------------------------------------------------------------------------
// Exact: every product and sum rounded separately, in the operation order of
// the method's definition (no contraction into FMA).  Used for FP32/BF16
// arithmetic.
template <class C> struct ArExact;
template <> struct ArExact<float> {
    __device__ static float mul(float a, float b) { return __fmul_rn(a, b); }
    __device__ static float add(float a, float b) { return __fadd_rn(a, b); }
    __device__ static float madd(float a, float b, float s) { return __fadd_rn(s, __fmul_rn(a, b)); }
    __device__ static float div(float a, float b) { return __fdiv_rn(a, b); }
};
template <> struct ArExact<double> {
    __device__ static double mul(double a, double b) { return __dmul_rn(a, b); }
    __device__ static double add(double a, double b) { return __dadd_rn(a, b); }
    __device__ static double madd(double a, double b, double s) { return __dadd_rn(s, __dmul_rn(a, b)); }
    __device__ static double div(double a, double b) { return __ddiv_rn(a, b); }
};
// Fused: every product added with one fused multiply-add, in the same order.
// Used for all FP64 arithmetic (the residual, operator application, GADI-FP64
// inner solves): the FP64 pipe, not memory, is the scarcer resource on this
// GPU.  Plain products and quotients are rounded separately.
struct ArFusedD {
    __device__ static double mul(double a, double b) { return __dmul_rn(a, b); }
    __device__ static double add(double a, double b) { return __dadd_rn(a, b); }
    __device__ static double madd(double a, double b, double s) { return fma(a, b, s); }
    __device__ static double div(double a, double b) { return __ddiv_rn(a, b); }
};
// FP32 (also the compute type of the BF16 inner solves) with fused
// multiply-add: one rounding per product-and-sum, and half the issue slots
// of a separate product and sum
struct ArFusedF {
    __device__ static float mul(float a, float b) { return __fmul_rn(a, b); }
    __device__ static float add(float a, float b) { return __fadd_rn(a, b); }
    __device__ static float madd(float a, float b, float s) { return __fmaf_rn(a, b, s); }
    __device__ static float div(float a, float b) { return __fdiv_rn(a, b); }
};
template <int PREC> struct InnerAr { using T = ArFusedF; };
template <> struct InnerAr<P_FP64> { using T = ArFusedD; };

// accumulator type of per-thread partial sums in the inner phases
template <int PREC> struct AccT { using T = float; };
template <> struct AccT<P_FP64> { using T = double; };

// Stencil operator at one element:  d x_c + c0 x_W + c1 x_E + c2 x_S + c3 x_N
// [+ c4 x_B + c5 x_T] [- e x_im for a real part, + e x_re for an imaginary
// part], summed in that order.
template <class A, class C, bool D3, bool CPLX>
__device__ __forceinline__ C stencil_at(C d, const C (&c)[6], C e, C xc, C xw, C xe, C xs, C xn,
                                        C xb, C xt, C xpart, bool is_im)
{
    C s = A::mul(d, xc);
    s = A::madd(c[0], xw, s);
    s = A::madd(c[1], xe, s);
    s = A::madd(c[2], xs, s);
    s = A::madd(c[3], xn, s);
    if constexpr (D3) {
        s = A::madd(c[4], xb, s);
        s = A::madd(c[5], xt, s);
    }
    if constexpr (CPLX) s = A::madd(is_im ? e : -e, xpart, s);
    return s;
}


// The complex class's imaginary diagonal at element v of the chunk that
// starts at element g (two elements per grid point): the scalar e of the
// coefficient set, or sign * T_i for a per-point T (`sig`, FP64) -- exact in
// the FP64 phases, rounded to u_s in the inner ones, as stored coefficients.
__device__ __forceinline__ double pt_e_exact(const double *sig, double sign, long long g, int v, double e)
{
    return sig ? sign * __ldg(sig + ((g + v) >> 1)) : e;
}
template <int PREC>
__device__ __forceinline__ typename Prec<PREC>::C pt_e_us(const double *sig, typename Prec<PREC>::C sign,
                                                          long long g, int v, typename Prec<PREC>::C e)
{
    using PT = Prec<PREC>;
    return sig ? sign * PT::ld(PT::from_f64(__ldg(sig + ((g + v) >> 1)))) : e;
}

// ---------------------------------------------------------------------------
// fields: the stencil input of a phase, computed from raw loads
// ---------------------------------------------------------------------------
// A field turns the raw 16-byte loads of N consecutive elements into N values
// of its type FT.  Raw data of a row are loaded PD rows before they are used,
// so the loads are split from the arithmetic: load<N>() fills a Raw<N>,
// value<N>() computes the field from it.  A zero Raw gives a zero field
// (Dirichlet value outside the grid).

// x + y in FP64 (the update fused into the residual); y may be absent
template <int PREC>
struct FieldX {
    using PT = Prec<PREC>;
    using S = typename PT::S;
    using FT = double;
    const double *x;
    const S *y;
    template <int N> struct Raw {
        double x[N];
        S y[N];
    };
    template <int N> __device__ void load(long long g, Raw<N> &r) const
    {
        VecIO<double, N>::load_ca(x + g, r.x);
        if (y) VecIO<S, N>::load_ca(y + g, r.y);
    }
    template <int N> __device__ void value(const Raw<N> &r, double (&o)[N]) const
    {
#pragma unroll
        for (int v = 0; v < N; v++) o[v] = y ? __dadd_rn(r.x[v], PT::to_f64(r.y[v])) : r.x[v];
    }
};

// fl_s(a), fl_s(b) as values of the compute type: for BF16 the two roundings
// by one instruction (the same round-to-nearest-even as one at a time)
template <int PREC, class C>
__device__ __forceinline__ void round_pair(C a, C b, C &ra, C &rb)
{
    using PT = Prec<PREC>;
    if constexpr (PREC == P_BF16) {
        f32x2_round_bf16(a, b, ra, rb);
    } else {
        ra = PT::ld(PT::st(a));
        rb = PT::ld(PT::st(b));
    }
}

// fl_s(src + beta p_old) (the CG direction update), or src on the first step
template <int PREC>
struct FieldDir {
    using PT = Prec<PREC>;
    using S = typename PT::S;
    using C = typename PT::C;
    using FT = C;
    using A = typename InnerAr<PREC>::T;
    const S *src, *pold;
    C beta;
    bool first;
    template <int N> struct Raw {
        S s[N], p[N];
    };
    template <int N> __device__ void load(long long g, Raw<N> &r) const
    {
        VecIO<S, N>::load_ca(src + g, r.s);
        if (!first) VecIO<S, N>::load_ca(pold + g, r.p);
    }
    template <int N> __device__ void value(const Raw<N> &r, C (&o)[N]) const
    {
        if constexpr (PREC == P_BF16 && N % 2 == 0) {
#pragma unroll
            for (int v = 0; v < N; v += 2) {
                if (first) {
                    o[v] = PT::ld(r.s[v]);
                    o[v + 1] = PT::ld(r.s[v + 1]);
                } else {
                    round_pair<PREC>(A::madd(beta, PT::ld(r.p[v]), PT::ld(r.s[v])),
                                     A::madd(beta, PT::ld(r.p[v + 1]), PT::ld(r.s[v + 1])), o[v], o[v + 1]);
                }
            }
        } else {
#pragma unroll
            for (int v = 0; v < N; v++)
                o[v] = first ? PT::ld(r.s[v]) : PT::ld(PT::st(A::madd(beta, PT::ld(r.p[v]), PT::ld(r.s[v]))));
        }
    }
    // shared-memory staging (march_smem): field vector k, whether it is read
    static constexpr int NF = 2;
    __device__ const S *vec(int k) const { return k == 0 ? src : pold; }
    __device__ bool used(int k) const { return k == 0 || !first; }
    template <int N> __device__ void from_smem(const S *c0, const S *c1, Raw<N> &r) const
    {
#pragma unroll
        for (int v = 0; v < N; v++) {
            r.s[v] = c0[v];
            r.p[v] = first ? S(0) : c1[v];
        }
    }
};

// a stored u_s vector, optionally scaled and re-rounded: fl_s(scale v)
template <int PREC, bool SCALE>
struct FieldLoad {
    using PT = Prec<PREC>;
    using S = typename PT::S;
    using C = typename PT::C;
    using FT = C;
    using A = typename InnerAr<PREC>::T;
    const S *src;
    C scale;
    template <int N> struct Raw {
        S s[N];
    };
    template <int N> __device__ void load(long long g, Raw<N> &r) const { VecIO<S, N>::load_ca(src + g, r.s); }
    template <int N> __device__ void value(const Raw<N> &r, C (&o)[N]) const
    {
        if constexpr (SCALE && PREC == P_BF16 && N % 2 == 0) {
#pragma unroll
            for (int v = 0; v < N; v += 2)
                round_pair<PREC>(A::mul(scale, PT::ld(r.s[v])), A::mul(scale, PT::ld(r.s[v + 1])), o[v], o[v + 1]);
        } else {
#pragma unroll
            for (int v = 0; v < N; v++) {
                if constexpr (SCALE) o[v] = PT::ld(PT::st(A::mul(scale, PT::ld(r.s[v]))));
                else o[v] = PT::ld(r.s[v]);
            }
        }
    }
    static constexpr int NF = 1;
    __device__ const S *vec(int) const { return src; }
    __device__ bool used(int) const { return true; }
    template <int N> __device__ void from_smem(const S *c0, const S *, Raw<N> &r) const
    {
#pragma unroll
        for (int v = 0; v < N; v++) r.s[v] = c0[v];
    }
};

// own-point inputs: NV vectors of type T at the output row
template <class T, int W, int NV>
struct OwnIn {
    T v[NV > 0 ? NV : 1][W];
};

template <class R, bool D3> struct YNbr {
    R s, n;
};
template <class R> struct YNbr<R, false> {};

// ---------------------------------------------------------------------------
// the marching sweep over a 2D or 3D grid
// ---------------------------------------------------------------------------
// A warp owns a strip of 32*W consecutive elements of a row (W per lane) and
// marches along the slowest axis (y in 2D, z in 3D) over a contiguous range
// of work units, keeping the field at rows m-1, m, m+1 in registers.  The raw
// loads of row m+PD+1 are issued while row m is computed (a ring of PD+1
// prefetched rows), so every warp keeps several rows of loads in flight.
// x neighbours come from warp shuffles; lanes 0 / 31 load the K elements just
// past the strip; 3D y neighbours are loaded with the row.  Outside the grid
// the field is zero (Dirichlet).  Work units are split evenly and contiguously
// over all warps of the grid.
template <class Ph, int W, int K, bool D3>
struct Slot {
    using F = typename Ph::Fld;
    typename F::template Raw<W> c;
    typename F::template Raw<K> hl, hr;
    typename Ph::Own o;
    YNbr<typename F::template Raw<W>, D3> y;
};

// Balanced contiguous split of `nunits` work units over the warps of a
// virtual grid, in 32-bit arithmetic (64-bit integer division is a long
// instruction sequence; the host keeps nunits below 2^31).  Warp w gets
// [w q + min(w, rem), ... + q + (w < rem)).
__device__ __forceinline__ void split_units(int nunits, VGrid vg, int &u0, int &u1)
{
    const int GW = (int)vg.nwarps(), gw = (int)vg.warp();
    const int q = nunits / GW, rem = nunits - q * GW;
    u0 = gw * q + min(gw, rem);
    u1 = u0 + q + (gw < rem ? 1 : 0);
}

// Load the raw data of row g into a slot.  Invalid rows (outside the grid)
// get a zero field; halo raws are written only for the lanes that use them
// (lane 0 / 31), own-point raws only for rows the warp outputs.
template <int W, int K, bool D3, class Ph>
__device__ __forceinline__ void load_slot(const Ph &ph, Slot<Ph, W, K, D3> &sl, bool valid, bool own,
                                          long long g, int lane, int e0, int ne, int yy, int ny)
{
    sl = Slot<Ph, W, K, D3>{};
    if (!valid) return;
    ph.f.template load<W>(g, sl.c);
    if (lane == 0 && e0 > 0) ph.f.template load<K>(g - K, sl.hl);
    if (lane == 31 && e0 + W < ne) ph.f.template load<K>(g + W, sl.hr);
    if (own) ph.load_own(g, sl.o);
    if constexpr (D3) {
        if (yy > 0) ph.f.template load<W>(g - ne, sl.y.s);
        if (yy + 1 < ny) ph.f.template load<W>(g + ne, sl.y.n);
    }
}

template <int W, int K, bool D3, int PD, class Ph, class ACC>
__device__ __forceinline__ void march(const Ph &ph, int ne, int ny, int nz, ACC &acc, VGrid vg)
{
    using FT = typename Ph::Fld::FT;
    using SL = Slot<Ph, W, K, D3>;
    const int lane = threadIdx.x & 31;
    const int nstrips = (ne + 32 * W - 1) / (32 * W);
    const int collen = D3 ? nz : ny;
    const long long mstride = D3 ? (long long)ne * ny : (long long)ne;
    // 2D: warps split (strip, row) units.  3D: blocks split (strip, y-tile, z)
    // units; the warps of a block take consecutive y rows of one tile and
    // march the same z range, so each warp's y-neighbour rows are the rows
    // its neighbour warps load at the same time (L1 hits).
    const int wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    const int nyt = D3 ? (ny + nwb - 1) / nwb : 1;
    const int ncols = D3 ? nstrips * nyt : nstrips;
    int u, u1;
    if constexpr (D3) {
        const int nb = vg.n, bi = vg.b, nu = ncols * collen;
        const int q = nu / nb, rem = nu - q * nb;
        u = bi * q + min(bi, rem);
        u1 = u + q + (bi < rem ? 1 : 0);
    } else {
        split_units(ncols * collen, vg, u, u1);
    }
    while (u < u1) {
        const int col = u / collen;
        const int m0 = u - col * collen;
        const int m1 = min(collen, m0 + (u1 - u));
        u += m1 - m0;
        const int strip = D3 ? col / nyt : col;
        const int yy = D3 ? (col - strip * nyt) * nwb + wib : 0;
        if (D3 && yy >= ny) continue; // past the last row of a partial tile
        const int e0 = strip * 32 * W + lane * W;
        const bool act = e0 < ne;
        const long long cbase = (D3 ? (long long)yy * ne : 0ll) + e0;

        typename Ph::Fld::template Raw<W> rdn{};
        if (act && m0 > 0) ph.f.template load<W>(cbase + (long long)(m0 - 1) * mstride, rdn);
        SL ring[PD + 1];
#pragma unroll
        for (int i = 0; i <= PD; i++) {
            const int m = m0 + i;
            load_slot<W, K, D3>(ph, ring[i], act && m < collen, m < m1, cbase + (long long)m * mstride, lane,
                                e0, ne, yy, ny);
        }
        FT dn[W], cu[W], up[W];
        ph.f.template value<W>(rdn, dn);
        ph.f.template value<W>(ring[0].c, cu);
        for (int m = m0; m < m1; ++m) {
            // ring[0] = row m, ring[1] = row m+1, ..., ring[PD] = row m+PD
            SL nxt;
            {
                const int mn = m + PD + 1;
                load_slot<W, K, D3>(ph, nxt, act && mn < collen, mn < m1, cbase + (long long)mn * mstride, lane,
                                    e0, ne, yy, ny);
            }
            ph.f.template value<W>(ring[PD >= 1 ? 1 : 0].c, up);
            if constexpr (PD == 0) ph.f.template value<W>(nxt.c, up);
            FT lh[K], rh[K];
#pragma unroll
            for (int k = 0; k < K; k++) {
                lh[k] = __shfl_up_sync(0xffffffffu, cu[W - K + k], 1);
                rh[k] = __shfl_down_sync(0xffffffffu, cu[k], 1);
            }
            if (lane == 0) ph.f.template value<K>(ring[0].hl, lh);
            if (lane == 31) ph.f.template value<K>(ring[0].hr, rh);
            FT w[W], e[W];
#pragma unroll
            for (int v = 0; v < W; v++) {
                w[v] = (v >= K) ? cu[v - K] : lh[v];
                e[v] = (v + K < W) ? cu[v + K] : rh[v + K - W];
            }
            if (act) {
                const long long g = cbase + (long long)m * mstride;
                if constexpr (D3) {
                    FT sy[W], ny_[W];
                    ph.f.template value<W>(ring[0].y.s, sy);
                    ph.f.template value<W>(ring[0].y.n, ny_);
                    ph.out(g, ring[0].o, cu, w, e, sy, ny_, dn, up, acc);
                } else {
                    ph.out(g, ring[0].o, cu, w, e, dn, up, dn, up, acc);
                }
            }
#pragma unroll
            for (int i = 0; i < PD; i++) ring[i] = ring[i + 1];
            ring[PD] = nxt;
#pragma unroll
            for (int v = 0; v < W; v++) {
                dn[v] = cu[v];
                cu[v] = up[v];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// the shared-memory-staged sweep (2D and complex 2D, 16-byte rows per lane)
// ---------------------------------------------------------------------------
// Same work split and arithmetic as march(), but a row's inputs reach the SM
// by asynchronous 16-byte copies (cp.async.cg) issued SMEM_PD rows ahead into
// a per-warp ring of shared-memory slots, so the prefetch depth costs no
// registers.  A slot holds, for every input vector of the phase, the 32
// lanes' 16-byte chunks, plus the chunk left of the strip (copied by lane 0)
// and right of it (lane 31) for each field vector.  Rows outside the grid and
// chunks past the row ends are zero-filled by the copy itself (source size 0).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool fill)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    const int n = fill ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

constexpr int SMEM_PD = 3;                         // rows copied ahead
constexpr int SMEM_NS = SMEM_PD + 2;               // slots per warp
constexpr int SMEM_SLOT = 4 * 32 * 16 + 4 * 16;    // <= 4 vectors, <= 2 field vectors
constexpr int SMEM_WARP = SMEM_NS * SMEM_SLOT;

// copy row m (element offset g of lane's chunk) of a phase into a slot
template <int W, class Ph>
__device__ __forceinline__ void smem_issue_row(const Ph &ph, unsigned char *slot, bool inrow, bool own, long long g,
                                               int lane, int e0, int ne)
{
    using F = typename Ph::Fld;
    using S = typename F::S;
    constexpr int NF = F::NF, NO = Ph::NO, NV = NF + NO;
    const bool act = e0 < ne;
#pragma unroll
    for (int k = 0; k < NF; k++) {
        if (!ph.f.used(k)) continue;
        const S *base = ph.f.vec(k);
        const bool ok = inrow && act;
        cp_async16(slot + k * 512 + lane * 16, ok ? (const void *)(base + g) : (const void *)base, ok);
        if (lane == 0) {
            const bool okl = inrow && act && e0 > 0;
            cp_async16(slot + NV * 512 + k * 16, okl ? (const void *)(base + g - W) : (const void *)base, okl);
        }
        if (lane == 31) {
            const bool okr = inrow && act && e0 + W < ne;
            cp_async16(slot + NV * 512 + (NF + k) * 16, okr ? (const void *)(base + g + W) : (const void *)base,
                       okr);
        }
    }
    if (own) {
#pragma unroll
        for (int k = 0; k < NO; k++) {
            if (!ph.own_used(k)) continue;
            const S *base = ph.own_vec(k);
            const bool ok = inrow && act;
            cp_async16(slot + (NF + k) * 512 + lane * 16, ok ? (const void *)(base + g) : (const void *)base, ok);
        }
    }
}

template <int W, int K, class Ph, class AT>
__device__ __forceinline__ void march_smem(const Ph &ph, int ne, int ny, AT (&acc)[2], unsigned char *wsm, VGrid vg)
{
    using F = typename Ph::Fld;
    using S = typename F::S;
    using FT = typename F::FT;
    constexpr int NF = F::NF, NO = Ph::NO, NV = NF + NO;
    static_assert(W * sizeof(S) == 16, "march_smem needs 16-byte lane chunks");
    static_assert(NV <= 4 && NF <= 2, "slot layout");
    const int lane = threadIdx.x & 31;
    const int nstrips = (ne + 32 * W - 1) / (32 * W);
    int u, u1;
    split_units(nstrips * ny, vg, u, u1);
    while (u < u1) {
        const int strip = u / ny;
        const int m0 = u - strip * ny;
        const int m1 = min(ny, m0 + (u1 - u));
        u += m1 - m0;
        const int e0 = strip * 32 * W + lane * W;
        const bool act = e0 < ne;
        const long long cbase = e0;
        // slot of row m: (m - m0 + 1) % SMEM_NS
        auto slot_of = [&](int m) { return wsm + ((m - m0 + 1) % SMEM_NS) * SMEM_SLOT; };
        for (int r = m0 - 1; r < m0 + SMEM_PD; ++r) {
            smem_issue_row<W>(ph, slot_of(r), r >= 0 && r < ny, r >= m0 && r < m1, cbase + (long long)r * ne,
                              lane, e0, ne);
            cp_async_commit();
        }
        FT dn[W], cu[W], up[W];
        for (int m = m0; m < m1; ++m) {
            {
                const int r = m + SMEM_PD;
                smem_issue_row<W>(ph, slot_of(r), r < ny, r < m1, cbase + (long long)r * ne, lane, e0, ne);
                cp_async_commit();
            }
            cp_async_wait<SMEM_PD - 1>(); // rows <= m + 1 have landed
            __syncwarp();
            typename F::template Raw<W> raw;
            if (m == m0) {
                const unsigned char *sd = slot_of(m0 - 1), *sc = slot_of(m0);
                ph.f.template from_smem<W>((const S *)(sd + lane * 16), (const S *)(sd + 512 + lane * 16), raw);
                ph.f.template value<W>(raw, dn);
                ph.f.template from_smem<W>((const S *)(sc + lane * 16), (const S *)(sc + 512 + lane * 16), raw);
                ph.f.template value<W>(raw, cu);
            }
            const unsigned char *sc = slot_of(m), *su = slot_of(m + 1);
            ph.f.template from_smem<W>((const S *)(su + lane * 16), (const S *)(su + 512 + lane * 16), raw);
            ph.f.template value<W>(raw, up);
            FT lh[K], rh[K];
#pragma unroll
            for (int k = 0; k < K; k++) {
                lh[k] = __shfl_up_sync(0xffffffffu, cu[W - K + k], 1);
                rh[k] = __shfl_down_sync(0xffffffffu, cu[k], 1);
            }
            if (lane == 0) {
                typename F::template Raw<K> rk;
                const unsigned char *h = sc + NV * 512;
                ph.f.template from_smem<K>((const S *)h + (W - K), (const S *)(h + 16) + (W - K), rk);
                ph.f.template value<K>(rk, lh);
            }
            if (lane == 31) {
                typename F::template Raw<K> rk;
                const unsigned char *h = sc + NV * 512 + NF * 16;
                ph.f.template from_smem<K>((const S *)h, (const S *)(h + 16), rk);
                ph.f.template value<K>(rk, rh);
            }
            FT w[W], e[W];
#pragma unroll
            for (int v = 0; v < W; v++) {
                w[v] = (v >= K) ? cu[v - K] : lh[v];
                e[v] = (v + K < W) ? cu[v + K] : rh[v + K - W];
            }
            if (act) {
                typename Ph::Own o;
                const S *oc[NO > 0 ? NO : 1];
#pragma unroll
                for (int k = 0; k < NO; k++) oc[k] = (const S *)(sc + (NF + k) * 512 + lane * 16);
                ph.own_from_smem(oc, o);
                ph.out(cbase + (long long)m * ne, o, cu, w, e, dn, up, dn, up, acc);
            }
            __syncwarp(); // every lane is done with row m's slot before it is refilled
#pragma unroll
            for (int v = 0; v < W; v++) {
                dn[v] = cu[v];
                cu[v] = up[v];
            }
        }
        cp_async_wait<0>();
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// the shared-memory-staged 3D sweep (16-byte rows per lane)
// ---------------------------------------------------------------------------
// The block's warps take the NWB consecutive y rows of one tile of a strip
// (as in march) and march z together, one plane of the tile per step.  Each
// step's inputs reach the SM by asynchronous 16-byte copies issued SM3_PD
// planes ahead into a block-wide ring of plane slots: per field vector the
// tile's rows plus the row below and above it (copied by the first and last
// warp), the x-halo chunks of each row (lanes 0 / 31), and the own-point
// vectors of each row.  A warp reads its y neighbours from the rows its
// neighbour warps copied, so every row crosses from memory to the SM once per
// phase, and the loads in flight cost shared memory instead of registers.
// One block barrier per step makes a plane's copies visible to every warp
// and frees the slot of the plane before it.  Outside the grid the copies
// zero-fill (Dirichlet).
constexpr int SM3_NWB = kThreads / 32;           // rows of a tile
#ifndef GADI_SM3_PD
#define GADI_SM3_PD 4
#endif
constexpr int SM3_PD = GADI_SM3_PD;              // planes copied ahead
constexpr int SM3_NS = SM3_PD + 1;               // plane slots
template <int NF, int NO>
struct Sm3Layout {
    static constexpr int ROW = 32 * 16;                              // a row's lane chunks
    static constexpr int FIELD = NF * (SM3_NWB + 2) * ROW;           // field rows
    static constexpr int HALO = NF * SM3_NWB * 2 * 16;               // x-halo chunks
    static constexpr int SLOT = FIELD + HALO + NO * SM3_NWB * ROW;   // + own rows
    // field vector k, tile row j (0: the row below the tile, NWB + 1: above)
    static constexpr int field(int k, int j) { return (k * (SM3_NWB + 2) + j) * ROW; }
    // x-halo chunk of field vector k at tile row w (0-based), side 0 left / 1 right
    static constexpr int halo(int k, int w, int side) { return FIELD + ((k * SM3_NWB + w) * 2 + side) * 16; }
    static constexpr int own(int k, int w) { return FIELD + HALO + (k * SM3_NWB + w) * ROW; }
};
// the largest slot of the inner phases: one field vector and three own-point
// vectors (CGNR's S2), above two field vectors and none (the fused direction)
constexpr int SM3_SLOT_MAX = Sm3Layout<1, 3>::SLOT > Sm3Layout<2, 0>::SLOT ? Sm3Layout<1, 3>::SLOT
                                                                           : Sm3Layout<2, 0>::SLOT;
constexpr int SM3_BYTES = SM3_NS * SM3_SLOT_MAX;

// copy plane p of the tile (rows yy0 - 1 .. yy0 + NWB) into a slot
template <int W, class Ph>
__device__ __forceinline__ void sm3_issue_plane(const Ph &ph, unsigned char *slot, int p, bool own, int nz,
                                                int ny, int ne, int yy0, int e0, int lane, int wib)
{
    using F = typename Ph::Fld;
    using S = typename F::S;
    using L = Sm3Layout<F::NF, Ph::NO>;
    const bool act = e0 < ne;
    const bool pin = p >= 0 && p < nz;
    const int yy = yy0 + wib;
    const long long g = ((long long)p * ny + yy) * ne + e0; // this warp's row
    const bool rin = pin && act && yy < ny;
#pragma unroll
    for (int k = 0; k < F::NF; k++) {
        if (!ph.f.used(k)) continue;
        const S *base = ph.f.vec(k);
        cp_async16(slot + L::field(k, wib + 1) + lane * 16, rin ? (const void *)(base + g) : (const void *)base, rin);
        if (lane == 0) {
            const bool ok = rin && e0 > 0;
            cp_async16(slot + L::halo(k, wib, 0), ok ? (const void *)(base + g - W) : (const void *)base, ok);
        }
        if (lane == 31) {
            const bool ok = rin && e0 + W < ne;
            cp_async16(slot + L::halo(k, wib, 1), ok ? (const void *)(base + g + W) : (const void *)base, ok);
        }
        if (wib == 0) { // the row below the tile
            const bool ok = pin && act && yy0 > 0;
            cp_async16(slot + L::field(k, 0) + lane * 16, ok ? (const void *)(base + g - ne) : (const void *)base,
                       ok);
        }
        if (wib == SM3_NWB - 1) { // the row above the tile
            const bool ok = pin && act && yy + 1 < ny;
            cp_async16(slot + L::field(k, SM3_NWB + 1) + lane * 16,
                       ok ? (const void *)(base + g + ne) : (const void *)base, ok);
        }
    }
    if (own) {
#pragma unroll
        for (int k = 0; k < Ph::NO; k++) {
            if (!ph.own_used(k)) continue;
            const S *base = ph.own_vec(k);
            cp_async16(slot + L::own(k, wib) + lane * 16, rin ? (const void *)(base + g) : (const void *)base, rin);
        }
    }
}

template <int W, int K, class Ph, class AT>
__device__ __forceinline__ void march3_smem(const Ph &ph, int ne, int ny, int nz, AT (&acc)[2], VGrid vg)
{
    extern __shared__ __align__(16) unsigned char gadi_dsmem[];
    unsigned char *const sm = gadi_dsmem;
    using F = typename Ph::Fld;
    using S = typename F::S;
    using FT = typename F::FT;
    using L = Sm3Layout<F::NF, Ph::NO>;
    static_assert(W * sizeof(S) == 16, "march3_smem needs 16-byte lane chunks");
    static_assert(K == 1, "the 3D class has one x neighbour per side");
    static_assert(L::SLOT <= SM3_SLOT_MAX, "slot layout");
    static_assert(SM3_PD >= 2, "the wait below keeps planes m+2.. in flight");
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nstrips = (ne + 32 * W - 1) / (32 * W);
    const int nyt = (ny + SM3_NWB - 1) / SM3_NWB;
    const int ncols = nstrips * nyt;
    // the block's contiguous share of the (strip, y-tile, z) units: the same
    // for all its warps, so every warp takes every step and every barrier
    int u, u1;
    {
        const int nb = vg.n, bi = vg.b, nu = ncols * nz;
        const int q = nu / nb, rem = nu - q * nb;
        u = bi * q + min(bi, rem);
        u1 = u + q + (bi < rem ? 1 : 0);
    }
    while (u < u1) {
        const int col = u / nz;
        const int m0 = u - col * nz;
        const int m1 = min(nz, m0 + (u1 - u));
        u += m1 - m0;
        const int strip = col / nyt;
        const int yy0 = (col - strip * nyt) * SM3_NWB;
        const int yy = yy0 + wib;
        const int e0 = strip * 32 * W + lane * W;
        const bool act = e0 < ne && yy < ny;
        const long long cbase = (long long)yy * ne + e0;
        const long long mstride = (long long)ne * ny;
        auto slot_of = [&](int p) { return sm + ((unsigned)(p - m0) % SM3_NS) * SM3_SLOT_MAX; };
        // plane m0 - 1 of this warp's row: loaded directly (only its centre
        // values are used)
        typename F::template Raw<W> raw{};
        if (act && m0 > 0) ph.f.template load<W>(cbase + (long long)(m0 - 1) * mstride, raw);
        FT dn[W], cu[W], up[W];
        ph.f.template value<W>(raw, dn);
        for (int p = m0; p < m0 + SM3_PD; ++p) {
            if (p <= m1) sm3_issue_plane<W>(ph, slot_of(p), p, p < m1, nz, ny, ne, yy0, e0, lane, wib);
            cp_async_commit();
        }
        for (int m = m0; m < m1; ++m) {
            cp_async_wait<SM3_PD - 2>(); // planes <= m + 1 of this thread have landed
            __syncthreads();             // ... of every thread; every warp is past step m - 1
            {
                const int p = m + SM3_PD; // into the slot of plane m - 1
                if (p <= m1) sm3_issue_plane<W>(ph, slot_of(p), p, p < m1, nz, ny, ne, yy0, e0, lane, wib);
                cp_async_commit();
            }
            const unsigned char *sc = slot_of(m), *su = slot_of(m + 1);
            auto row = [&](const unsigned char *sl, int j, int k) {
                return (const S *)(sl + L::field(k, j) + lane * 16);
            };
            if (m == m0) {
                ph.f.template from_smem<W>(row(sc, wib + 1, 0), row(sc, wib + 1, F::NF - 1), raw);
                ph.f.template value<W>(raw, cu);
            }
            ph.f.template from_smem<W>(row(su, wib + 1, 0), row(su, wib + 1, F::NF - 1), raw);
            ph.f.template value<W>(raw, up);
            FT lh[K], rh[K];
            lh[0] = __shfl_up_sync(0xffffffffu, cu[W - 1], 1);
            rh[0] = __shfl_down_sync(0xffffffffu, cu[0], 1);
            if (lane == 0) {
                typename F::template Raw<K> rk;
                ph.f.template from_smem<K>((const S *)(sc + L::halo(0, wib, 0)) + (W - K),
                                           (const S *)(sc + L::halo(F::NF - 1, wib, 0)) + (W - K), rk);
                ph.f.template value<K>(rk, lh);
            }
            if (lane == 31) {
                typename F::template Raw<K> rk;
                ph.f.template from_smem<K>((const S *)(sc + L::halo(0, wib, 1)),
                                           (const S *)(sc + L::halo(F::NF - 1, wib, 1)), rk);
                ph.f.template value<K>(rk, rh);
            }
            FT w[W], e[W];
#pragma unroll
            for (int v = 0; v < W; v++) {
                w[v] = (v >= K) ? cu[v - K] : lh[v];
                e[v] = (v + K < W) ? cu[v + K] : rh[v + K - W];
            }
            if (act) {
                FT sy[W], ny_[W];
                ph.f.template from_smem<W>(row(sc, wib, 0), row(sc, wib, F::NF - 1), raw);
                ph.f.template value<W>(raw, sy);
                ph.f.template from_smem<W>(row(sc, wib + 2, 0), row(sc, wib + 2, F::NF - 1), raw);
                ph.f.template value<W>(raw, ny_);
                typename Ph::Own o;
                const S *oc[Ph::NO > 0 ? Ph::NO : 1];
#pragma unroll
                for (int k = 0; k < Ph::NO; k++) oc[k] = (const S *)(sc + L::own(k, wib) + lane * 16);
                ph.own_from_smem(oc, o);
                ph.out(cbase + (long long)m * mstride, o, cu, w, e, sy, ny_, dn, up, acc);
            }
#pragma unroll
            for (int v = 0; v < W; v++) {
                dn[v] = cu[v];
                cu[v] = up[v];
            }
        }
        cp_async_wait<0>();
        __syncthreads(); // every warp is done with the slots before the next column reuses them
    }
}

// ---------------------------------------------------------------------------
// stencil phases (field + own-point inputs + output)
// ---------------------------------------------------------------------------
// R: x_out = x + y, r = b - A x_out (FP64), r_s = fl_s(r); sums ||r||^2 and
// ||r_s||^2.  With b == nullptr it is the operator application x_out = A x.
// DD: r in double-FP64 (u_r ~ u^2, Sec. 3.1): starting from b, every term
// -a_j x_j enters as an exact product p + pe (fused multiply-add) added by
// TwoSum, the errors summed alongside (the Dot2 scheme of Ogita, Rump &
// Oishi 2005), in the stencil's order (centre, W, E, S, N[, B, T][, the
// complex coupling]); r = hi + lo after a final TwoSum.
__device__ __forceinline__ void dd_sub_term(double &hi, double &lo, double a, double x)
{
    double p, pe, q;
    two_prod(-a, x, p, pe);
    two_sum(hi, p, hi, q);
    lo = __dadd_rn(lo, __dadd_rn(q, pe));
}

// x * 2^k is x with k added to its exponent field when x is normal and the
// result stays normal (then exact); zero, subnormal, infinite and NaN x or a
// result out of the normal range need the multiplication
__device__ __forceinline__ bool pow2_shift_ok(double x, int k)
{
    const int ex = (int)((__double_as_longlong(x) >> 52) & 0x7ff);
    return ex != 0 && ex != 0x7ff && ex + k >= 1 && ex + k <= 0x7fe;
}

template <int PREC, int W, int K, bool D3, bool DD = false>
struct PhResidual {
    using PT = Prec<PREC>;
    using S = typename PT::S;
    using A = ArFusedD; // FP64 products accumulated by fused multiply-add
    using Fld = FieldX<PREC>;
    using Own = OwnIn<double, W, 1>;
    Fld f;
    double *xo;
    const double *b;
    double *rout;
    S *rs;
    Coef7<double> cf;
    double *rlo; // DD: low parts of r (nullable)
    const double *sig = nullptr; // complex class: per-point T (null: cf.e)
    double esign = 1.0;
    int dpow2 = kNoPow2; // cf.d = 2^dpow2 (see mul_pow2), else kNoPow2
    __device__ void load_own(long long g, Own &o) const
    {
        if (b) VecIO<double, W>::load(b + g, o.v[0]);
    }
    template <class AT>
    __device__ void out(long long g, const Own &o, const double (&c)[W], const double (&w)[W],
                        const double (&e)[W], const double (&s)[W], const double (&n)[W],
                        const double (&bb)[W], const double (&t)[W], AT (&acc)[2]) const
    {
        double r[W], rl[W];
        if constexpr (DD) {
#pragma unroll
            for (int v = 0; v < W; v++) {
                double hi = o.v[0][v], lo = 0.0;
                dd_sub_term(hi, lo, cf.d, c[v]);
                dd_sub_term(hi, lo, cf.c[0], w[v]);
                dd_sub_term(hi, lo, cf.c[1], e[v]);
                dd_sub_term(hi, lo, cf.c[2], s[v]);
                dd_sub_term(hi, lo, cf.c[3], n[v]);
                if constexpr (D3) {
                    dd_sub_term(hi, lo, cf.c[4], bb[v]);
                    dd_sub_term(hi, lo, cf.c[5], t[v]);
                }
                if constexpr (K == 2) {
                    const double ev = pt_e_exact(sig, esign, g, v, cf.e);
                    dd_sub_term(hi, lo, (v & 1) ? ev : -ev, c[v ^ 1]);
                }
                two_sum(hi, lo, r[v], rl[v]);
            }
        } else {
            double ax[W];
            // with a power-of-two centre (the 2D 5-point Laplacian's 4) the
            // product cf.d x is an exponent shift, exact and bit-identical,
            // taken on the integer pipe when the whole warp's points allow it
            bool shift = false;
            if constexpr (K == 1) {
                bool ok = dpow2 != kNoPow2;
#pragma unroll
                for (int v = 0; v < W; v++) ok = ok && pow2_shift_ok(c[v], dpow2);
                shift = __all_sync(__activemask(), ok); // out() runs on the strip's active lanes
            }
            if (shift) {
#pragma unroll
                for (int v = 0; v < W; v++) {
                    double q = __longlong_as_double(__double_as_longlong(c[v]) + ((long long)dpow2 << 52));
                    q = fma(cf.c[0], w[v], q);
                    q = fma(cf.c[1], e[v], q);
                    q = fma(cf.c[2], s[v], q);
                    q = fma(cf.c[3], n[v], q);
                    if constexpr (D3) {
                        q = fma(cf.c[4], bb[v], q);
                        q = fma(cf.c[5], t[v], q);
                    }
                    ax[v] = q;
                }
            } else {
#pragma unroll
                for (int v = 0; v < W; v++)
                    ax[v] = stencil_at<A, double, D3, K == 2>(cf.d, cf.c,
                                                              K == 2 ? pt_e_exact(sig, esign, g, v, cf.e) : 0.0,
                                                              c[v], w[v], e[v], s[v], n[v], bb[v], t[v],
                                                              c[v ^ (K - 1)], (v & 1) != 0);
            }
            if (b == nullptr) { // operator application: xo = Op x
                VecIO<double, W>::store(xo + g, ax);
                return;
            }
#pragma unroll
            for (int v = 0; v < W; v++) r[v] = __dsub_rn(o.v[0][v], ax[v]);
        }
        S so[W];
        // ||r_s||^2 (the start of CG on H, in the inner solve's compute type)
        // is summed per thread in FP32 like every dot product of the inner
        // solves, off the FP64 pipe that carries the residual itself; the
        // per-thread partial travels in the low 32 bits of acc[1] (the high
        // half stays zero) and is widened for the grid-wide sum.
        float s2 = __int_as_float(__double2loint(acc[1]));
#pragma unroll
        for (int v = 0; v < W; v++) {
            acc[0] = fma(r[v], r[v], acc[0]);
            if constexpr (DD) so[v] = PT::from_f64x2(r[v], rl[v]);
            else so[v] = PT::from_f64(r[v]);
            const float sf = PT::ld(so[v]);
            s2 = __fmaf_rn(sf, sf, s2);
        }
        acc[1] = __hiloint2double(0, __float_as_int(s2));
        VecIO<double, W>::store(xo + g, c);
        VecIO<S, W>::store(rs + g, so);
        if (rout) VecIO<double, W>::store(rout + g, r);
        if constexpr (DD)
            if (rlo) VecIO<double, W>::store(rlo + g, rl);
    }
};

// H1: p = fl_s(r + beta p_old); sum p.(H p).  With STORE_Q (all-FP64 inner
// arithmetic, where the FP64 pipe is the bottleneck) H p is also written out
// so that H2 needs no stencil.
template <int PREC, int W, int K, bool D3, bool STORE_Q>
struct PhH1 {
    using PT = Prec<PREC>;
    using S = typename PT::S;
    using C = typename PT::C;
    using A = typename InnerAr<PREC>::T;
    using Fld = FieldDir<PREC>;
    using Own = OwnIn<S, W, 0>;
    Fld f;
    S *pnew;
    S *qout;
    Coef7<C> h;
    __device__ void load_own(long long, Own &) const {}
    static constexpr int NO = 0;
    __device__ const S *own_vec(int) const { return nullptr; }
    __device__ bool own_used(int) const { return false; }
    __device__ void own_from_smem(const S *const *, Own &) const {}
    template <class AT>
    __device__ void out(long long g, const Own &, const C (&c)[W], const C (&w)[W], const C (&e)[W],
                        const C (&s)[W], const C (&n)[W], const C (&b)[W], const C (&t)[W], AT (&acc)[2]) const
    {
        S ps[W], qs[W];
#pragma unroll
        for (int v = 0; v < W; v++) {
            const C q = stencil_at<A, C, D3, false>(h.d, h.c, C(0), c[v], w[v], e[v], s[v], n[v], b[v], t[v],
                                                    C(0), false);
            acc[0] += (AT)c[v] * (AT)q;
            ps[v] = PT::st(c[v]);
            qs[v] = PT::st(q);
        }
        VecIO<S, W>::store(pnew + g, ps);
        if constexpr (STORE_Q) VecIO<S, W>::store(qout + g, qs);
    }
};

// H2: z = fl_s(z + a p), r = fl_s(r - a H p) with H p recomputed; sum r.r
template <int PREC, int W, int K, bool D3>
struct PhH2 {
    using PT = Prec<PREC>;
    using S = typename PT::S;
    using C = typename PT::C;
    using A = typename InnerAr<PREC>::T;
    using Fld = FieldLoad<PREC, false>;
    using Own = OwnIn<S, W, 2>; // z, r
    Fld f;
    S *z, *r;
    C a;
    bool first;
    Coef7<C> h;
    __device__ void load_own(long long g, Own &o) const
    {
        if (!first) VecIO<S, W>::load(z + g, o.v[0]);
        VecIO<S, W>::load(r + g, o.v[1]);
    }
    static constexpr int NO = 2;
    __device__ const S *own_vec(int k) const { return k == 0 ? z : r; }
    __device__ bool own_used(int k) const { return k == 1 || !first; }
    __device__ void own_from_smem(const S *const *c, Own &o) const
    {
#pragma unroll
        for (int v = 0; v < W; v++) {
            o.v[0][v] = first ? S(0) : c[0][v];
            o.v[1][v] = c[1][v];
        }
    }
    template <class AT>
    __device__ void out(long long g, const Own &o, const C (&c)[W], const C (&w)[W], const C (&e)[W],
                        const C (&s)[W], const C (&n)[W], const C (&b)[W], const C (&t)[W], AT (&acc)[2]) const
    {
        S zv[W], rv[W];
#pragma unroll
        for (int v = 0; v < W; v++) {
            const C q = stencil_at<A, C, D3, false>(h.d, h.c, C(0), c[v], w[v], e[v], s[v], n[v], b[v], t[v],
                                                    C(0), false);
            zv[v] = PT::st(first ? A::mul(a, c[v]) : A::madd(a, c[v], PT::ld(o.v[0][v])));
            rv[v] = PT::st(A::madd(-a, q, PT::ld(o.v[1][v])));
            const C rr = PT::ld(rv[v]);
            acc[0] += (AT)rr * (AT)rr;
        }
        VecIO<S, W>::store(z + g, zv);
        VecIO<S, W>::store(r + g, rv);
    }
};

// p.(H p) with p already stored (the 3D form of H1: a pointwise p update
// first, so the stencil pass reads p instead of recomputing it from r and
// p_old at every neighbour row)
template <int PREC, int W, int K, bool D3, bool STORE_Q = false>
struct PhPHp {
    using PT = Prec<PREC>;
    using S = typename PT::S;
    using C = typename PT::C;
    using A = typename InnerAr<PREC>::T;
    using Fld = FieldLoad<PREC, false>;
    using Own = OwnIn<S, W, 0>;
    Fld f;
    Coef7<C> h;
    S *qout; // STORE_Q: H p written out for a pointwise H2
    __device__ void load_own(long long, Own &) const {}
    static constexpr int NO = 0;
    __device__ const S *own_vec(int) const { return nullptr; }
    __device__ bool own_used(int) const { return false; }
    __device__ void own_from_smem(const S *const *, Own &) const {}
    template <class AT>
    __device__ void out(long long g, const Own &, const C (&c)[W], const C (&w)[W], const C (&e)[W],
                        const C (&s)[W], const C (&n)[W], const C (&b)[W], const C (&t)[W], AT (&acc)[2]) const
    {
        S qs[W];
#pragma unroll
        for (int v = 0; v < W; v++) {
            const C q = stencil_at<A, C, D3, false>(h.d, h.c, C(0), c[v], w[v], e[v], s[v], n[v], b[v], t[v],
                                                    C(0), false);
            acc[0] += (AT)c[v] * (AT)q;
            qs[v] = PT::st(q);
        }
        if constexpr (STORE_Q) VecIO<S, W>::store(qout + g, qs);
    }
};

// u = fl_s(S p) with p already stored (the 3D form of S1); sum u.u
template <int PREC, int W, int K, bool D3>
struct PhSu {
    using PT = Prec<PREC>;
    using S = typename PT::S;
    using C = typename PT::C;
    using A = typename InnerAr<PREC>::T;
    using Fld = FieldLoad<PREC, false>;
    using Own = OwnIn<S, W, 0>;
    Fld f;
    S *u;
    Coef7<C> sc;
    const double *sig = nullptr; // complex class: per-point T (null: sc.e)
    __device__ void load_own(long long, Own &) const {}
    static constexpr int NO = 0;
    __device__ const S *own_vec(int) const { return nullptr; }
    __device__ bool own_used(int) const { return false; }
    __device__ void own_from_smem(const S *const *, Own &) const {}
    template <class AT>
    __device__ void out(long long g, const Own &, const C (&c)[W], const C (&w)[W], const C (&e)[W],
                        const C (&s)[W], const C (&n)[W], const C (&b)[W], const C (&t)[W], AT (&acc)[2]) const
    {
        S us[W];
#pragma unroll
        for (int v = 0; v < W; v++) {
            const C q = stencil_at<A, C, D3, K == 2>(sc.d, sc.c, K == 2 ? pt_e_us<PREC>(sig, C(+1), g, v, sc.e) : C(0),
                                                     c[v], w[v], e[v], s[v], n[v], b[v], t[v], c[v ^ (K - 1)],
                                                     (v & 1) != 0);
            us[v] = PT::st(q);
            const C uu = PT::ld(us[v]);
            acc[0] += (AT)uu * (AT)uu;
        }
        VecIO<S, W>::store(u + g, us);
    }
};

// S0: t = fl_s(S^T fl_s(gamma z)); sum t.t
template <int PREC, int W, int K, bool D3>
struct PhS0 {
    using PT = Prec<PREC>;
    using S = typename PT::S;
    using C = typename PT::C;
    using A = typename InnerAr<PREC>::T;
    using Fld = FieldLoad<PREC, true>;
    using Own = OwnIn<S, W, 0>;
    Fld f;
    S *t;
    Coef7<C> st;
    const double *sig = nullptr; // complex class: per-point T (null: st.e)
    __device__ void load_own(long long, Own &) const {}
    static constexpr int NO = 0;
    __device__ const S *own_vec(int) const { return nullptr; }
    __device__ bool own_used(int) const { return false; }
    __device__ void own_from_smem(const S *const *, Own &) const {}
    template <class AT>
    __device__ void out(long long g, const Own &, const C (&c)[W], const C (&w)[W], const C (&e)[W],
                        const C (&s)[W], const C (&n)[W], const C (&b)[W], const C (&tt)[W], AT (&acc)[2]) const
    {
        S to[W];
#pragma unroll
        for (int v = 0; v < W; v++) {
            const C q = stencil_at<A, C, D3, K == 2>(st.d, st.c, K == 2 ? pt_e_us<PREC>(sig, C(-1), g, v, st.e) : C(0), c[v], w[v], e[v], s[v], n[v], b[v], tt[v],
                                                     c[v ^ (K - 1)], (v & 1) != 0);
            to[v] = PT::st(q);
            const C qq = PT::ld(to[v]);
            acc[0] += (AT)qq * (AT)qq;
        }
        VecIO<S, W>::store(t + g, to);
    }
};

// S1: p = fl_s(t + beta p_old), u = fl_s(S p); sum u.u
template <int PREC, int W, int K, bool D3>
struct PhS1 {
    using PT = Prec<PREC>;
    using S = typename PT::S;
    using C = typename PT::C;
    using A = typename InnerAr<PREC>::T;
    using Fld = FieldDir<PREC>;
    using Own = OwnIn<S, W, 0>;
    Fld f;
    S *pnew, *u;
    Coef7<C> sc;
    const double *sig = nullptr; // complex class: per-point T (null: sc.e)
    __device__ void load_own(long long, Own &) const {}
    static constexpr int NO = 0;
    __device__ const S *own_vec(int) const { return nullptr; }
    __device__ bool own_used(int) const { return false; }
    __device__ void own_from_smem(const S *const *, Own &) const {}
    template <class AT>
    __device__ void out(long long g, const Own &, const C (&c)[W], const C (&w)[W], const C (&e)[W],
                        const C (&s)[W], const C (&n)[W], const C (&b)[W], const C (&t)[W], AT (&acc)[2]) const
    {
        S ps[W], us[W];
#pragma unroll
        for (int v = 0; v < W; v++) {
            const C q = stencil_at<A, C, D3, K == 2>(sc.d, sc.c, K == 2 ? pt_e_us<PREC>(sig, C(+1), g, v, sc.e) : C(0), c[v], w[v], e[v], s[v], n[v], b[v], t[v],
                                                     c[v ^ (K - 1)], (v & 1) != 0);
            us[v] = PT::st(q);
            const C uu = PT::ld(us[v]);
            acc[0] += (AT)uu * (AT)uu;
            ps[v] = PT::st(c[v]);
        }
        VecIO<S, W>::store(pnew + g, ps);
        VecIO<S, W>::store(u + g, us);
    }
};

// S2: y = fl_s(y + a p), t = fl_s(t - a S^T u); sum t.t
template <int PREC, int W, int K, bool D3>
struct PhS2 {
    using PT = Prec<PREC>;
    using S = typename PT::S;
    using C = typename PT::C;
    using A = typename InnerAr<PREC>::T;
    using Fld = FieldLoad<PREC, false>;
    using Own = OwnIn<S, W, 3>; // p, y, t
    Fld f;
    const S *p;
    S *y, *t;
    C a;
    bool first;
    Coef7<C> st;
    const double *sig = nullptr; // complex class: per-point T (null: st.e)
    __device__ void load_own(long long g, Own &o) const
    {
        VecIO<S, W>::load(p + g, o.v[0]);
        if (!first) VecIO<S, W>::load(y + g, o.v[1]);
        VecIO<S, W>::load(t + g, o.v[2]);
    }
    static constexpr int NO = 3;
    __device__ const S *own_vec(int k) const { return k == 0 ? p : (k == 1 ? y : t); }
    __device__ bool own_used(int k) const { return k != 1 || !first; }
    __device__ void own_from_smem(const S *const *c, Own &o) const
    {
#pragma unroll
        for (int v = 0; v < W; v++) {
            o.v[0][v] = c[0][v];
            o.v[1][v] = first ? S(0) : c[1][v];
            o.v[2][v] = c[2][v];
        }
    }
    template <class AT>
    __device__ void out(long long g, const Own &o, const C (&c)[W], const C (&w)[W], const C (&e)[W],
                        const C (&s)[W], const C (&n)[W], const C (&b)[W], const C (&tt)[W], AT (&acc)[2]) const
    {
        S yv[W], tv[W];
#pragma unroll
        for (int v = 0; v < W; v++) {
            const C q = stencil_at<A, C, D3, K == 2>(st.d, st.c, K == 2 ? pt_e_us<PREC>(sig, C(-1), g, v, st.e) : C(0), c[v], w[v], e[v], s[v], n[v], b[v], tt[v],
                                                     c[v ^ (K - 1)], (v & 1) != 0);
            const C pp = PT::ld(o.v[0][v]);
            yv[v] = PT::st(first ? A::mul(a, pp) : A::madd(a, pp, PT::ld(o.v[1][v])));
            tv[v] = PT::st(A::madd(-a, q, PT::ld(o.v[2][v])));
            const C t2 = PT::ld(tv[v]);
            acc[0] += (AT)t2 * (AT)t2;
        }
        VecIO<S, W>::store(y + g, yv);
        VecIO<S, W>::store(t + g, tv);
    }
};

// ---------------------------------------------------------------------------
// stencil implementation of the phase interface
// ---------------------------------------------------------------------------
// the coefficient set k (0 H, 1 S, 2 S^T) of the launch in compute type C
template <class C> __device__ __forceinline__ const Coef7<C> &coef_set(const Params &p, int k);
template <> __device__ __forceinline__ const Coef7<float> &coef_set<float>(const Params &p, int k)
{
    return k == 0 ? p.hf : (k == 1 ? p.sf : p.tf);
}
template <> __device__ __forceinline__ const Coef7<double> &coef_set<double>(const Params &p, int k)
{
    return k == 0 ? p.hd : (k == 1 ? p.sd : p.td);
}

// DD: the residual phase in double-FP64 (u_r ~ u^2); a separate
// instantiation, so the FP64-residual kernels carry none of its code.
// CMODE: how the H, S, S^T coefficients are held -- 0: copies of the
// launch parameters' sets, 1: read from the launch parameters where they are
// used (the tensor-memory kernel, whose registers are short), 2: converted
// from the FP64 coefficients once (the 2D streaming kernel, measured fastest
// so at 4096^2).
template <int KIND, int PREC, int WI, int WR, bool DD = false, int CMODE = 0>
struct StencilImpl {
    using PT = Prec<PREC>;
    using S = typename PT::S;
    using C = typename PT::C;
    using A = typename InnerAr<PREC>::T;
    using AT = typename AccT<PREC>::T;
    static constexpr int K = (KIND == K_C2D5) ? 2 : 1;
    static constexpr bool D3 = (KIND == K_3D7);
    static constexpr bool STORE_Q = (PREC == P_FP64);
    static constexpr int PD = D3 ? 1 : 1; // rows prefetched ahead (register ring)
    // 2D rows with 16-byte lane chunks go through the shared-memory-staged sweep
    static constexpr bool USE_SMEM = GADI_SMEM_SWEEP && !D3 && (WI * sizeof(S) == 16);
    // 3D FP32 and BF16 rows with 16-byte lane chunks: the block-wide plane
    // ring (march3_smem).  At 512^3 it took a CG iteration on H from 1.07 to
    // 0.77 ms (FP32) and 0.59 to 0.52 ms (BF16, the direction update fused,
    // see SPLIT_P), and the first 300 outer iterations of the solve from
    // 19.4 to 15.1 ms (FP32) and 8.1 to 7.9 ms (BF16) each.  FP64 inner
    // solves, bound by the FP64 pipe, ran 7 % slower per CG iteration with it
    // and keep the register ring.
        static constexpr bool USE_SMEM3 = GADI_SMEM3 && D3 && PREC != P_FP64 && (WI * sizeof(S) == 16);
    // rows the residual's register ring prefetches: none in the kernels with
    // the plane ring, whose inner phases otherwise push the kernel's
    // allocation into spills inside the residual's loop (a BF16 solve then
    // ran 10.0 instead of 7.9 ms per outer iteration at 512^3, FP32 16.0
    // instead of 15.1), in the 3D FP64 kernel (spills 220 -> 16 bytes, CGNR
    // iteration 5.87 -> 5.47 ms) and in the 2D tensor-memory kernel (CMODE 1;
    // 2048^2 solve 1.149 -> 1.143 s); the residual is bound by the FP64 pipe,
    // and its step time did not change (4.46 ms FP32, 4.65 ms BF16, 3.78 ms
    // FP64 at 512^3)
    static constexpr int RPD = (USE_SMEM3 || (D3 && PREC == P_FP64) || CMODE == 1) ? 0 : PD;
    static constexpr int DSMEM = USE_SMEM ? (kThreads / 32) * SMEM_WARP : (USE_SMEM3 ? SM3_BYTES : 0);
    const Params &P;
    VGrid vg;
    int ne, ny, nz;
    Coef7<double> ca;
    // H, S and S^T in the compute type (see CMODE)
    using CoefSet = std::conditional_t<CMODE == 1, const Coef7<C> &, Coef7<C>>;
    CoefSet ch, cs, ct;

    __device__ StencilImpl(const Params &p, VGrid g)
        : P(p), vg(g), ch(coef_set<C>(p, 0)), cs(coef_set<C>(p, 1)), ct(coef_set<C>(p, 2))
    {
        ne = p.nx * K;
        ny = p.ny;
        nz = D3 ? p.nz : 1;
        if constexpr (CMODE == 2) {
            ch.d = (C)p.co.h_d; ch.e = C(0);
            cs.d = (C)p.co.s_d; cs.e = (C)p.co.s_e;
            ct.d = (C)p.co.t_d; ct.e = (C)p.co.t_e;
#pragma unroll
            for (int k = 0; k < 6; k++) {
                ch.c[k] = (C)p.co.h_c[k];
                cs.c[k] = (C)p.co.s_c[k];
                ct.c[k] = (C)p.co.t_c[k];
            }
        }
        ca.d = p.co.a_d; ca.e = p.co.a_e;
#pragma unroll
        for (int k = 0; k < 6; k++) ca.c[k] = p.co.a_c[k];
    }

    __device__ static unsigned char *warp_smem()
    {
        extern __shared__ __align__(16) unsigned char gadi_dsmem[];
        return gadi_dsmem + (threadIdx.x >> 5) * SMEM_WARP;
    }
    // run a phase over the grid with the sweep this instantiation uses
    template <class Ph>
    __device__ void sweep(const Ph &ph, AT (&acc)[2]) const
    {
        acc[0] = acc[1] = AT(0);
        if constexpr (USE_SMEM) march_smem<WI, K>(ph, ne, ny, acc, warp_smem(), vg);
        else if constexpr (USE_SMEM3) march3_smem<WI, K>(ph, ne, ny, nz, acc, vg);
        else march<WI, K, D3, PD>(ph, ne, ny, nz, acc, vg);
    }

    __device__ void residual(const double *xin, const S *y, double *xout, double (&acc)[2]) const
    {
        double a[2] = {0.0, 0.0}; // a[1]: the FP32 partial of the r_s norm in its low 32 bits
        PhResidual<PREC, WR, K, D3, DD> ph{{xin, y}, xout, P.b, P.r_out, (S *)P.r, ca, P.r_lo_out, P.sig, P.sig_a};
        ph.dpow2 = P.ad_pow2;
        march<WR, K, D3, RPD>(ph, ne, ny, nz, a, vg);
        acc[0] = a[0];
        acc[1] = (double)__int_as_float(__double2hiint(a[1])) + (double)__int_as_float(__double2loint(a[1]));
    }
    __device__ void apply(const double *x, double *yout) const
    {
        PhResidual<PREC, WR, K, D3> ph{{x, nullptr}, yout, nullptr, nullptr, nullptr, ca, nullptr, P.sig, P.sig_a};
        ph.dpow2 = P.ad_pow2;
        double a[2] = {0.0, 0.0};
        march<WR, K, D3, RPD>(ph, ne, ny, nz, a, vg);
    }
    __device__ void h1(bool first, C beta, const S *pold, S *pnew, AT (&acc)[2]) const
    {
        PhH1<PREC, WI, K, D3, STORE_Q> ph;
        ph.f.src = (const S *)P.r; ph.f.pold = pold; ph.f.beta = beta; ph.f.first = first;
        ph.pnew = pnew; ph.qout = (S *)P.u; ph.h = ch;
        sweep(ph, acc);
    }
    __device__ void h2(bool first, C a_, const S *p, AT (&acc)[2]) const
    {
        if constexpr (STORE_Q) {
            // pointwise: z += a p, r -= a q with q = H p stored by H1
            using V = VecIO<S, WI>;
            S *z = (S *)P.z, *r = (S *)P.r;
            const S *q = (const S *)P.u;
            AT s = AT(0);
            const long long nv = P.nelem / WI;
            for (long long i = vg.tid(); i < nv; i += vg.nthreads()) {
                const long long g = i * WI;
                S pv[WI], qv[WI], zv[WI], rv[WI];
                V::load(p + g, pv);
                V::load(q + g, qv);
                V::load(r + g, rv);
                if (!first) V::load(z + g, zv);
#pragma unroll
                for (int v = 0; v < WI; v++) {
                    zv[v] = first ? A::mul(a_, pv[v]) : A::madd(a_, pv[v], zv[v]);
                    rv[v] = A::madd(-a_, qv[v], rv[v]);
                    s += (AT)rv[v] * (AT)rv[v];
                }
                V::store(z + g, zv);
                V::store(r + g, rv);
            }
            acc[0] = s;
            acc[1] = AT(0);
        } else {
            PhH2<PREC, WI, K, D3> ph;
            ph.f.src = p; ph.f.scale = C(1);
            ph.z = (S *)P.z; ph.r = (S *)P.r; ph.a = a_; ph.first = first; ph.h = ch;
            sweep(ph, acc);
        }
    }
    __device__ void s0(C gamma, AT (&acc)[2]) const
    {
        PhS0<PREC, WI, K, D3> ph;
        ph.f.src = (const S *)P.z; ph.f.scale = gamma; ph.t = (S *)P.r; ph.st = ct; ph.sig = P.sig;
        sweep(ph, acc);
    }
    __device__ void s1(bool first, C beta, const S *pold, S *pnew, AT (&acc)[2]) const
    {
        PhS1<PREC, WI, K, D3> ph;
        ph.f.src = (const S *)P.r; ph.f.pold = pold; ph.f.beta = beta; ph.f.first = first;
        ph.pnew = pnew; ph.u = (S *)P.u; ph.sc = cs; ph.sig = P.sig;
        sweep(ph, acc);
    }
    // 3D FP64 (the register ring): the direction update p = fl_s(src + beta
    // p_old) (p = src at first) as its own pointwise pass (src = P.r: the CG
    // residual r or the CGNR residual t), then the stencil pass on the stored
    // p.  Measured at 512^3 / 320^3 on the register ring: 5-6 % faster per
    // outer iteration for BF16 and FP64, slower for FP32 (whose fused pass
    // recomputes p at the neighbour rows more cheaply than an extra pass over
    // memory costs).  On the plane ring the fused update is faster for BF16
    // too (CG iteration 0.52 vs 0.56 ms at 512^3).
    static constexpr bool SPLIT_P = D3 && !USE_SMEM3 && (PREC == P_BF16 || PREC == P_FP64);
    __device__ void p_update(bool first, C beta, const S *pold, S *pnew) const
    {
        using A2 = typename InnerAr<PREC>::T;
        const S *src = (const S *)P.r;
        const long long nch = P.nelem / WI;
        for (long long ch_ = vg.tid(); ch_ < nch; ch_ += vg.nthreads()) {
            const long long g = ch_ * WI;
            S sv[WI], pv[WI];
            VecIO<S, WI>::load(src + g, sv);
            if (!first) VecIO<S, WI>::load(pold + g, pv);
#pragma unroll
            for (int v = 0; v < WI; v++)
                pv[v] = first ? sv[v] : PT::st(A2::madd(beta, PT::ld(pv[v]), PT::ld(sv[v])));
            VecIO<S, WI>::store(pnew + g, pv);
        }
    }
    __device__ void h1_split(const S *p, AT (&acc)[2]) const
    {
        PhPHp<PREC, WI, K, D3, STORE_Q> ph;
        ph.f.src = p; ph.f.scale = C(1); ph.h = ch; ph.qout = (S *)P.u;
        sweep(ph, acc);
    }
    __device__ void s1_split(const S *p, AT (&acc)[2]) const
    {
        PhSu<PREC, WI, K, D3> ph;
        ph.f.src = p; ph.f.scale = C(1); ph.u = (S *)P.u; ph.sc = cs; ph.sig = P.sig;
        sweep(ph, acc);
    }
    __device__ void s2(bool first, C a_, const S *p, AT (&acc)[2]) const
    {
        PhS2<PREC, WI, K, D3> ph;
        ph.f.src = (const S *)P.u; ph.f.scale = C(1); ph.p = p; ph.y = (S *)P.y; ph.t = (S *)P.r;
        ph.a = a_; ph.first = first; ph.st = ct; ph.sig = P.sig;
        sweep(ph, acc);
    }
    // ---- SM-resident H-solve (2D real class, FP32/BF16, 16-byte chunks) ----
    // Block b owns rows [ya, yb) (a balanced split of the ny rows over the
    // group's blocks) and keeps p of those rows plus one halo row on each side
    // in shared memory, as floats holding u_s-rounded values, for the whole
    // CG solve.  r and z stay in global memory (L2) and are streamed with no
    // dependency chain.  The halo rows of p are recomputed by this block from
    // the neighbour's rows of r with the same rounded operations as their
    // owner: p_0 = r_0 and p_j = fl_s(r_j + beta p_{j-1}), where p_{j-1} of a
    // halo row is what this block put in the halo slot one iteration before.
    // By induction the halo equals the owner's rows bit for bit, so blocks
    // exchange nothing but r, and an iteration keeps its two grid barriers.
    static constexpr bool RES_OK = (KIND == K_2D5) && (PREC != P_FP64) && (WI * sizeof(S) == 16);
    __device__ void res_rows(int &ya, int &yb) const
    {
        ya = vg.b * ny / vg.n;
        yb = (vg.b + 1) * ny / vg.n;
    }
    __device__ static float *res_smem()
    {
        extern __shared__ __align__(16) unsigned char gadi_dsmem[];
        return reinterpret_cast<float *>(gadi_dsmem);
    }
    // chunks of W elements a thread loads before it uses any of them: the
    // global loads of the resident phases have no dependency chain, so U of
    // them are kept in flight per thread instead of one per row
    static constexpr int RES_U = PREC == P_BF16 ? 2 : 4;
    // rows of z and r the H2 march keeps in flight ahead of the one it updates
    static constexpr int RES_PD = PREC == P_BF16 ? 3 : 4;
    // the first RES_PD rows of z and r of a thread's first column pass: the
    // H2 march starts from them, and they can be loaded while the barrier
    // of the p.(Hp) sum is still open (they are this block's own rows)
    struct ResRing {
        S z[RES_PD][WI], r[RES_PD][WI];
    };
    // p = fl_s(r + beta p_old) on the slab and its halo rows, then the sum of
    // p.(H p) over the slab
    __device__ GADI_RES_FN void h1_res(int j, C beta, AT (&acc)[2]) const
    {
        if constexpr (RES_OK) {
            constexpr int W = WI, U = RES_U;
            using A2 = typename InnerAr<PREC>::T;
            int ya, yb;
            res_rows(ya, yb);
            const int R = yb - ya, nxw = ne / W;
            // rows ya-1 .. yb that exist in the grid (the halo slot of a grid
            // edge stays zero: it is cleared once, at j = 0)
            const int rlo = ya > 0 ? -1 : 0, rhi = yb < ny ? R : R - 1;
            const int i_lo = (rlo + 1) * nxw, i_hi = (rhi + 2) * nxw;
            float *sp = res_smem();
            const S *r = (const S *)P.r;
            const bool first = j == 0;
            if (first) {
                if (ya == 0)
                    for (int i = threadIdx.x; i < ne; i += blockDim.x) sp[i] = 0.f;
                if (yb == ny)
                    for (int i = threadIdx.x; i < ne; i += blockDim.x) sp[(size_t)(R + 1) * ne + i] = 0.f;
            }
            // chunk i covers elements [i W, i W + W) counted from row ya - 1
            // (i >= nxw whenever ya = 0, so every offset used is >= 0)
            const long long off0 = (long long)(ya - 1) * ne;
            const int step = U * (int)blockDim.x;
            for (int i0 = i_lo + threadIdx.x; i0 < i_hi; i0 += step) {
                const S *rp = r + (off0 + (long long)i0 * W);
                float *pp = sp + (size_t)i0 * W;
                S rv[U][W];
#pragma unroll
                for (int u = 0; u < U; u++)
                    if (i0 + u * (int)blockDim.x < i_hi) VecIO<S, W>::load(rp + (size_t)u * blockDim.x * W, rv[u]);
#pragma unroll
                for (int u = 0; u < U; u++) {
                    if (i0 + u * (int)blockDim.x >= i_hi) break;
                    float4 *d4 = reinterpret_cast<float4 *>(pp + (size_t)u * blockDim.x * W);
#pragma unroll
                    for (int v = 0; v < W; v += 4) {
                        float4 t;
                        if (first) {
                            t = make_float4(PT::ld(rv[u][v]), PT::ld(rv[u][v + 1]), PT::ld(rv[u][v + 2]),
                                            PT::ld(rv[u][v + 3]));
                        } else {
                            t = d4[v / 4];
                            round_pair<PREC>(A2::madd(beta, t.x, PT::ld(rv[u][v])),
                                             A2::madd(beta, t.y, PT::ld(rv[u][v + 1])), t.x, t.y);
                            round_pair<PREC>(A2::madd(beta, t.z, PT::ld(rv[u][v + 2])),
                                             A2::madd(beta, t.w, PT::ld(rv[u][v + 3])), t.z, t.w);
                        }
                        d4[v / 4] = t;
                    }
                }
            }
            __syncthreads();
            AT a = AT(0);
            ResRing none;
            res_march<false>(false, C(0), a, none, false);
            acc[0] = a;
            acc[1] = AT(0);
        } else {
            acc[0] = acc[1] = AT(0);
        }
    }
    // load the ring the H2 march starts from (see ResRing)
    __device__ GADI_RES_FN void h2_res_pre(bool first, ResRing &q) const
    {
        if constexpr (RES_OK) {
            int ya, yb;
            res_rows(ya, yb);
            const ResMap m = res_map(yb - ya, ne / WI);
            res_ring_load(first, m, ya, m.cx0, q);
        }
    }
    // z = fl_s(z + a p), r = fl_s(r - a H p) on the slab, p from shared
    // memory; q: the ring of the first column pass, already loaded
    __device__ GADI_RES_FN void h2_res(bool first, C a_, AT (&acc)[2], ResRing &q) const
    {
        if constexpr (RES_OK) {
            AT s = AT(0);
            res_march<true>(first, a_, s, q, true);
            acc[0] = s;
            acc[1] = AT(0);
        } else {
            acc[0] = acc[1] = AT(0);
        }
    }
    // Thread -> (column chunk, row part) map of the column marches.  With at
    // least as many W-element chunks per row as threads, thread t takes the
    // chunks t, t + blockDim, ... down all slab rows; with fewer, the slab
    // rows are split into blockDim / nxw parts and thread t takes chunk
    // t % nxw of part t / nxw.  Every thread makes the same number of steps
    // (rmax per column pass; steps past its rows touch no memory) so that
    // the warp shuffles always see the whole warp.
    struct ResMap {
        int cx0, ncp, r0, r1, rmax;
        bool act;
    };
    __device__ ResMap res_map(int R, int nxw) const
    {
        ResMap m;
        const int t = threadIdx.x, nt = blockDim.x;
        if (nxw >= nt) {
            m.cx0 = t;
            m.ncp = (nxw + nt - 1) / nt;
            m.r0 = 0;
            m.r1 = m.rmax = R;
            m.act = true;
        } else {
            const int np = nt / nxw, part = t / nxw;
            m.cx0 = t - part * nxw;
            m.ncp = 1;
            m.act = part < np;
            m.r0 = m.act ? part * R / np : 0;
            m.r1 = m.act ? (part + 1) * R / np : 0;
            m.rmax = (R + np - 1) / np;
        }
        return m;
    }
    // One march of every thread's column chunks down its slab rows.  p comes
    // from shared memory: the rows below and at the current one stay in
    // registers, one new row is read per step, and the west / east
    // neighbours come from the adjacent lanes (shared memory only at a warp
    // or part edge).  UPD = false: acc += p.(H p).  UPD = true: the H2
    // update of z and r, whose rows are prefetched PD steps ahead, and
    // acc += r.r.
    __device__ void res_ring_load(bool first, const ResMap &m, int ya, int cx, ResRing &q) const
    {
        if (!m.act || cx >= ne / WI) return;
        const size_t o = (size_t)(ya + m.r0) * ne + (size_t)cx * WI;
        const S *zp = (const S *)P.z + o, *rp = (const S *)P.r + o;
#pragma unroll
        for (int k = 0; k < RES_PD; k++) {
            if (m.r0 + k < m.r1) {
                if (!first) VecIO<S, WI>::load(zp + (size_t)k * ne, q.z[k]);
                VecIO<S, WI>::load(rp + (size_t)k * ne, q.r[k]);
            }
        }
    }
    // pre: the ring of column pass 0 is already in q (UPD only)
    template <bool UPD>
    __device__ void res_march(bool first, C a_, AT &acc, ResRing &q, bool pre) const
    {
        constexpr int W = WI, PD = RES_PD;
        using A2 = typename InnerAr<PREC>::T;
        int ya, yb;
        res_rows(ya, yb);
        const int R = yb - ya, nxw = ne / W;
        const float *sp = res_smem();
        const ResMap m = res_map(R, nxw);
        const int lane = threadIdx.x & 31;
        for (int cp = 0; cp < m.ncp; ++cp) {
            const int cx = m.cx0 + cp * (int)blockDim.x;
            const bool col = m.act && cx < nxw;
            const int x0 = col ? cx * W : 0;
            // the adjacent lanes hold chunks cx - 1 and cx + 1 of the same rows
            const bool lsh = lane > 0 && cx > 0, rsh = lane < 31 && cx + 1 < nxw;
            const bool xlo = x0 > 0, xhi = x0 + W < ne;
            // walking pointers: the next shared-memory row to read (the row
            // below the current one), and z / r at the current row
            const float *up_p = sp + (size_t)(m.r0 + 2) * ne + x0;
            S *zp = (S *)P.z + ((size_t)(ya + m.r0) * ne + x0);
            S *rp = (S *)P.r + ((size_t)(ya + m.r0) * ne + x0);
            S (&zq)[PD][W] = q.z;
            S (&rq)[PD][W] = q.r;
            if constexpr (UPD) {
                if (!(pre && cp == 0)) res_ring_load(first, m, ya, cx, q);
            }
            float dn[W], c[W], up[W];
#pragma unroll
            for (int v = 0; v < W; v++) dn[v] = c[v] = up[v] = 0.f;
            if (col) {
                res_row<W>(up_p - 2 * (size_t)ne, dn);
                res_row<W>(up_p - (size_t)ne, c);
            }
            int left = col ? m.r1 - m.r0 : 0; // rows still to do in this column
            for (int i0 = 0; i0 < m.rmax; i0 += PD) {
#pragma unroll
                for (int k = 0; k < PD; k++) {
                    if (i0 + k >= m.rmax) break; // the same for every thread
                    const bool ok = left > 0;
                    if (ok) res_row<W>(up_p, up);
                    float cl = __shfl_up_sync(0xffffffffu, c[W - 1], 1);
                    float cr = __shfl_down_sync(0xffffffffu, c[0], 1);
                    if (ok) {
                        if (!lsh) cl = xlo ? up_p[-(ptrdiff_t)ne - 1] : 0.f;
                        if (!rsh) cr = xhi ? up_p[-(ptrdiff_t)ne + W] : 0.f;
                        S zv[W], rv[W];
#pragma unroll
                        for (int v = 0; v < W; v++) {
                            const float w = v > 0 ? c[v - 1] : cl, e = v + 1 < W ? c[v + 1] : cr;
                            const C q = stencil_at<A2, C, false, false>(ch.d, ch.c, C(0), c[v], w, e, dn[v], up[v],
                                                                        C(0), C(0), C(0), false);
                            if constexpr (UPD) {
                                zv[v] = PT::st(first ? A2::mul(a_, c[v]) : A2::madd(a_, c[v], PT::ld(zq[k][v])));
                                rv[v] = PT::st(A2::madd(-a_, q, PT::ld(rq[k][v])));
                                const C t = PT::ld(rv[v]);
                                acc += (AT)t * (AT)t;
                            } else {
                                acc += (AT)c[v] * (AT)q;
                            }
                        }
                        if constexpr (UPD) {
                            VecIO<S, W>::store(zp, zv);
                            VecIO<S, W>::store(rp, rv);
                            if (left > PD) { // refill this slot with the row PD steps ahead
                                if (!first) VecIO<S, W>::load(zp + (size_t)PD * ne, zq[k]);
                                VecIO<S, W>::load(rp + (size_t)PD * ne, rq[k]);
                            }
                        }
                    }
                    --left;
                    up_p += ne;
                    zp += ne;
                    rp += ne;
#pragma unroll
                    for (int v = 0; v < W; v++) {
                        dn[v] = c[v];
                        c[v] = up[v];
                    }
                }
            }
        }
    }
    // W floats of a shared-memory row (16-byte aligned)
    template <int W>
    __device__ static void res_row(const float *p, float (&o)[W])
    {
        const float4 *p4 = reinterpret_cast<const float4 *>(p);
#pragma unroll
        for (int v = 0; v < W; v += 4) {
            const float4 t = p4[v / 4];
            o[v] = t.x; o[v + 1] = t.y; o[v + 2] = t.z; o[v + 3] = t.w;
        }
    }

    // ---- z and r in tensor memory ----
    // The TMEM variant of the resident H-solve also keeps z and r of the
    // block's own rows on chip for the whole CG solve: each thread stores
    // its march chunks (column pass cp, step s -> slot cp * rmax + s) in
    // TMEM, z in the slot's first four columns and r in the next four (16
    // bytes each).  Global memory then sees only what other blocks need: r
    // of the slab's first and last row (the neighbours' halo) every
    // iteration, and z once, when the solve ends (all rows; only the first
    // and last when the resident S-solve follows, which takes the rest from
    // TMEM).  Same arithmetic as the L2 variant, so both give the same bits.
    static constexpr int TM_COLS = 512 / (kThreads / 128); // TMEM columns per warp
    static constexpr int TM_SLOTS = TM_COLS / 8;            // chunks of z and r per thread
    static constexpr bool TM_OK = RES_OK && (kThreads % 128) == 0 && TM_SLOTS >= 1;
    unsigned tm = 0; // TMEM base address of the block's allocation (512 columns)
    __device__ unsigned tm_addr(int slot, int which) const
    {
        const int w = threadIdx.x >> 5;
        return tm + ((unsigned)((w & 3) * 32) << 16) + (unsigned)((w >> 2) * TM_COLS + slot * 8 + which * 4);
    }
    // true if every thread's chunks fit its TMEM columns (the host checks the
    // same before it picks this variant)
    __device__ bool tm_fits() const
    {
        int ya, yb;
        res_rows(ya, yb);
        const ResMap m = res_map(yb - ya, ne / WI);
        return m.ncp * m.rmax <= TM_SLOTS;
    }
    template <int W>
    __device__ static void to_words(const S (&v)[W], unsigned (&w)[4])
    {
        static_assert(W * sizeof(S) == 16, "16-byte chunks");
        memcpy(w, v, 16);
    }
    template <int W>
    __device__ static void from_words(const unsigned (&w)[4], S (&v)[W])
    {
        memcpy(v, w, 16);
    }
    // p = fl_s(r + beta p) (p = r at j = 0) for one 16-byte chunk of p in
    // shared memory, as in h1_res
    template <int W>
    __device__ static void p_chunk(bool first, C beta, const S (&rv)[W], float *pp)
    {
        using A2 = typename InnerAr<PREC>::T;
        float4 *d4 = reinterpret_cast<float4 *>(pp);
#pragma unroll
        for (int v = 0; v < W; v += 4) {
            float4 t;
            if (first) {
                t = make_float4(PT::ld(rv[v]), PT::ld(rv[v + 1]), PT::ld(rv[v + 2]), PT::ld(rv[v + 3]));
            } else {
                t = d4[v / 4];
                round_pair<PREC>(A2::madd(beta, t.x, PT::ld(rv[v])), A2::madd(beta, t.y, PT::ld(rv[v + 1])), t.x,
                                 t.y);
                round_pair<PREC>(A2::madd(beta, t.z, PT::ld(rv[v + 2])), A2::madd(beta, t.w, PT::ld(rv[v + 3])), t.z,
                                 t.w);
            }
            d4[v / 4] = t;
        }
    }
    // p update and p.(H p), r of the own rows from TMEM (at j = 0 from
    // global memory, then kept), the halo rows from the neighbours' r
    __device__ GADI_RES_FN void h1_tm(int j, C beta, AT (&acc)[2]) const
    {
        if constexpr (TM_OK) {
            constexpr int W = WI, U = 4;
            int ya, yb;
            res_rows(ya, yb);
            const int R = yb - ya, nxw = ne / W;
            float *sp = res_smem();
            const S *r = (const S *)P.r;
            const bool first = j == 0;
            if (first) {
                if (ya == 0)
                    for (int i = threadIdx.x; i < ne; i += blockDim.x) sp[i] = 0.f;
                if (yb == ny)
                    for (int i = threadIdx.x; i < ne; i += blockDim.x) sp[(size_t)(R + 1) * ne + i] = 0.f;
            }
            // halo rows ya - 1 and yb (smem rows 0 and R + 1): the loads of a
            // thread's first HU chunks are issued before the own rows' work
            // and used after it
            constexpr int HU = 2;
            S hv[HU][W];
            int hc[HU];
#pragma unroll
            for (int u = 0; u < HU; u++) {
                const int i = (int)threadIdx.x + u * (int)blockDim.x;
                hc[u] = -1;
                if (i < 2 * nxw) {
                    const bool lo = i < nxw;
                    if (!(lo ? ya == 0 : yb == ny)) {
                        hc[u] = i;
                        VecIO<S, W>::load(r + ((long long)(lo ? ya - 1 : yb) * ne + (long long)(lo ? i : i - nxw) * W),
                                          hv[u]);
                    }
                }
            }
            // own rows, in the march's thread map
            const ResMap m = res_map(R, nxw);
            for (int cp = 0; cp < m.ncp; ++cp) {
                const int cx = m.cx0 + cp * (int)blockDim.x;
                const bool col = m.act && cx < nxw;
                const int x0 = col ? cx * W : 0;
                const int sb = cp * m.rmax;
                for (int s0 = 0; s0 < m.rmax; s0 += U) {
                    unsigned w[U][4];
#pragma unroll
                    for (int u = 0; u < U; u++) w[u][0] = w[u][1] = w[u][2] = w[u][3] = 0u;
                    if (first) {
                        S rv[U][W];
#pragma unroll
                        for (int u = 0; u < U; u++) {
                            if (col && m.r0 + s0 + u < m.r1)
                                VecIO<S, W>::load(r + ((size_t)(ya + m.r0 + s0 + u) * ne + x0), rv[u]);
                            else
                                for (int v = 0; v < W; v++) rv[u][v] = PT::st(C(0));
                        }
#pragma unroll
                        for (int u = 0; u < U; u++) {
                            to_words<W>(rv[u], w[u]);
                            if (s0 + u < m.rmax) tmem_st4(tm_addr(sb + s0 + u, 1), w[u]);
                        }
                    } else {
#pragma unroll
                        for (int u = 0; u < U; u++)
                            if (s0 + u < m.rmax) tmem_ld4(tm_addr(sb + s0 + u, 1), w[u]);
                        tmem_wait_ld<U>(w);
                    }
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        if (col && m.r0 + s0 + u < m.r1) {
                            S rv[W];
                            from_words<W>(w[u], rv);
                            p_chunk<W>(first, beta, rv, sp + (size_t)(m.r0 + s0 + u + 1) * ne + x0);
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < HU; u++) {
                if (hc[u] >= 0) {
                    const bool lo = hc[u] < nxw;
                    p_chunk<W>(first, beta, hv[u], sp + (size_t)(lo ? 0 : R + 1) * ne + (size_t)(lo ? hc[u] : hc[u] - nxw) * W);
                }
            }
            for (int i = (int)threadIdx.x + HU * (int)blockDim.x; i < 2 * nxw; i += blockDim.x) {
                const bool lo = i < nxw;
                if (lo ? ya == 0 : yb == ny) continue;
                const int c = lo ? i : i - nxw, row = lo ? -1 : R;
                S rv[W];
                VecIO<S, W>::load(r + ((long long)(ya + row) * ne + (long long)c * W), rv);
                p_chunk<W>(first, beta, rv, sp + (size_t)(row + 1) * ne + (size_t)c * W);
            }
            if (first) tmem_wait_st();
            __syncthreads();
            AT a = AT(0);
            ResRing none;
            res_march<false>(false, C(0), a, none, false);
            acc[0] = a;
            acc[1] = AT(0);
        } else {
            acc[0] = acc[1] = AT(0);
        }
    }
    // z = fl_s(z + a p), r = fl_s(r - a H p) with z and r in TMEM; r of the
    // slab's first and last row also to global memory (the neighbours' halo)
    __device__ GADI_RES_FN void h2_tm(bool first, C a_, AT (&acc)[2]) const
    {
        if constexpr (TM_OK) {
            constexpr int W = WI;
            using A2 = typename InnerAr<PREC>::T;
            int ya, yb;
            res_rows(ya, yb);
            const int R = yb - ya, nxw = ne / W;
            const float *sp = res_smem();
            const ResMap m = res_map(R, nxw);
            const int lane = threadIdx.x & 31;
            AT s2 = AT(0);
            for (int cp = 0; cp < m.ncp; ++cp) {
                const int cx = m.cx0 + cp * (int)blockDim.x;
                const bool col = m.act && cx < nxw;
                const int x0 = col ? cx * W : 0;
                const bool lsh = lane > 0 && cx > 0, rsh = lane < 31 && cx + 1 < nxw;
                const bool xlo = x0 > 0, xhi = x0 + W < ne;
                const float *up_p = sp + (size_t)(m.r0 + 2) * ne + x0;
                S *rg = (S *)P.r + ((size_t)(ya + m.r0) * ne + x0);
                const int sb = cp * m.rmax;
                unsigned w[2][4]; // z, r of the current step
#pragma unroll
                for (int k = 0; k < 2; k++) w[k][0] = w[k][1] = w[k][2] = w[k][3] = 0u;
                if (!first) tmem_ld4(tm_addr(sb, 0), w[0]);
                tmem_ld4(tm_addr(sb, 1), w[1]);
                float dn[W], c[W], up[W];
#pragma unroll
                for (int v = 0; v < W; v++) dn[v] = c[v] = up[v] = 0.f;
                if (col) {
                    res_row<W>(up_p - 2 * (size_t)ne, dn);
                    res_row<W>(up_p - (size_t)ne, c);
                }
                int left = col ? m.r1 - m.r0 : 0;
                for (int st = 0; st < m.rmax; ++st) {
                    const bool ok = left > 0;
                    if (ok) res_row<W>(up_p, up);
                    float cl = __shfl_up_sync(0xffffffffu, c[W - 1], 1);
                    float cr = __shfl_down_sync(0xffffffffu, c[0], 1);
                    C q[W];
#pragma unroll
                    for (int v = 0; v < W; v++) q[v] = C(0);
                    if (ok) {
                        if (!lsh) cl = xlo ? up_p[-(ptrdiff_t)ne - 1] : 0.f;
                        if (!rsh) cr = xhi ? up_p[-(ptrdiff_t)ne + W] : 0.f;
#pragma unroll
                        for (int v = 0; v < W; v++) {
                            const float wv = v > 0 ? c[v - 1] : cl, ev = v + 1 < W ? c[v + 1] : cr;
                            q[v] = stencil_at<A2, C, false, false>(ch.d, ch.c, C(0), c[v], wv, ev, dn[v], up[v], C(0),
                                                                  C(0), C(0), false);
                        }
                    }
                    tmem_wait_ld<2>(w);
                    S zv[W], rv[W];
                    from_words<W>(w[0], zv);
                    from_words<W>(w[1], rv);
                    if (ok) {
#pragma unroll
                        for (int v = 0; v < W; v++) {
                            zv[v] = PT::st(first ? A2::mul(a_, c[v]) : A2::madd(a_, c[v], PT::ld(zv[v])));
                            rv[v] = PT::st(A2::madd(-a_, q[v], PT::ld(rv[v])));
                            const C t = PT::ld(rv[v]);
                            s2 += (AT)t * (AT)t;
                        }
                        const int row = m.r0 + st;
                        if ((row == 0 && ya > 0) || (row == R - 1 && yb < ny)) VecIO<S, W>::store(rg, rv);
                    }
                    to_words<W>(zv, w[0]);
                    to_words<W>(rv, w[1]);
                    tmem_st4(tm_addr(sb + st, 0), w[0]);
                    tmem_st4(tm_addr(sb + st, 1), w[1]);
                    if (st + 1 < m.rmax) {
                        if (!first) tmem_ld4(tm_addr(sb + st + 1, 0), w[0]);
                        tmem_ld4(tm_addr(sb + st + 1, 1), w[1]);
                    }
                    --left;
                    up_p += ne;
                    rg += ne;
#pragma unroll
                    for (int v = 0; v < W; v++) {
                        dn[v] = c[v];
                        c[v] = up[v];
                    }
                }
            }
            tmem_wait_st();
            acc[0] = s2;
            acc[1] = AT(0);
        } else {
            acc[0] = acc[1] = AT(0);
        }
    }
    // one TMEM set of the own rows (which: 0 z / y, 1 r / t) to global
    // memory at dst; edges: only the rows the neighbours' halo needs
    // (edge_rows 1: the slab's first and last row; 2: its first two and last
    // two)
    __device__ void tm_flush(int which, S *dst, int edge_rows) const
    {
        if constexpr (TM_OK) {
            constexpr int W = WI, U = 4;
            int ya, yb;
            res_rows(ya, yb);
            const int R = yb - ya, nxw = ne / W;
            const ResMap m = res_map(R, nxw);
            for (int cp = 0; cp < m.ncp; ++cp) {
                const int cx = m.cx0 + cp * (int)blockDim.x;
                const bool col = m.act && cx < nxw;
                const int x0 = col ? cx * W : 0;
                const int sb = cp * m.rmax;
                for (int s0 = 0; s0 < m.rmax; s0 += U) {
                    unsigned w[U][4];
#pragma unroll
                    for (int u = 0; u < U; u++) w[u][0] = w[u][1] = w[u][2] = w[u][3] = 0u;
#pragma unroll
                    for (int u = 0; u < U; u++)
                        if (s0 + u < m.rmax) tmem_ld4(tm_addr(sb + s0 + u, which), w[u]);
                    tmem_wait_ld<U>(w);
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        const int row = m.r0 + s0 + u;
                        if (col && row < m.r1 && (edge_rows == 0 || row < edge_rows || row >= R - edge_rows)) {
                            S zv[W];
                            from_words<W>(w[u], zv);
                            VecIO<S, W>::store(dst + ((size_t)(ya + row) * ne + x0), zv);
                        }
                    }
                }
            }
        }
    }
    __device__ void h_flush_tm(bool edges_only) const { tm_flush(0, (S *)P.z, edges_only ? 1 : 0); }

    // ---- CGNR on S resident: p in shared memory, t and y in TMEM ----
    // The TMEM kernel's S-solve for blocks of two rows or more.  The slab
    // holds p (during s0: g = fl_s(gamma z)) of the rows ya - 2 .. yb + 1
    // (slot = row - ya + 2): u = fl_s(S p) is never stored but recomputed
    // where it is needed, from p with the owner's operations, so the S^T u
    // of a slab row needs p two rows out.  The halo rows of p are
    // recomputed from the neighbours' t (p = fl_s(t + beta p_old), the
    // induction of the H-solve); every block publishes t of its first two
    // and last two rows.  t takes the TMEM slots of r, y those of z.  Same
    // operations in the same order as the streaming phases PhS0-PhS2.
    __device__ bool s_edge(int row, int R, int ya, int yb) const
    {
        return (row < 2 && ya > 0) || (row >= R - 2 && yb < ny);
    }
    // s0: g = fl_s(gamma z) on the slab (halo rows from the neighbours'
    // published z; own rows from TMEM if z_tm, else from global memory),
    // then t = fl_s(S^T g), acc = t.t
    __device__ GADI_RES_FN void s0_tm(C gamma, bool z_tm, AT (&acc)[2]) const
    {
        if constexpr (TM_OK) {
            constexpr int W = WI, U = 4;
            using A2 = typename InnerAr<PREC>::T;
            int ya, yb;
            res_rows(ya, yb);
            const int R = yb - ya, nxw = ne / W;
            float *sp = res_smem();
            // slab rows outside the grid hold zeros (g and p vanish there)
            if (ya == 0)
                for (int i = threadIdx.x; i < 2 * ne; i += blockDim.x) sp[i] = 0.f;
            if (yb == ny)
                for (int i = threadIdx.x; i < 2 * ne; i += blockDim.x) sp[(size_t)(R + 2) * ne + i] = 0.f;
            const S *z = (const S *)P.z;
            for (int i = threadIdx.x; i < 2 * nxw; i += blockDim.x) {
                const bool lo = i < nxw;
                if (lo ? ya == 0 : yb == ny) continue;
                const int c = lo ? i : i - nxw, row = lo ? -1 : R;
                S zv[W];
                VecIO<S, W>::load(z + ((long long)(ya + row) * ne + (long long)c * W), zv);
                g_chunk<W>(gamma, zv, sp + (size_t)(row + 2) * ne + (size_t)c * W);
            }
            const ResMap m = res_map(R, nxw);
            for (int cp = 0; cp < m.ncp; ++cp) {
                const int cx = m.cx0 + cp * (int)blockDim.x;
                const bool col = m.act && cx < nxw;
                const int x0 = col ? cx * W : 0;
                const int sb = cp * m.rmax;
                for (int s0 = 0; s0 < m.rmax; s0 += U) {
                    unsigned w[U][4];
#pragma unroll
                    for (int u = 0; u < U; u++) w[u][0] = w[u][1] = w[u][2] = w[u][3] = 0u;
                    if (z_tm) {
#pragma unroll
                        for (int u = 0; u < U; u++)
                            if (s0 + u < m.rmax) tmem_ld4(tm_addr(sb + s0 + u, 0), w[u]);
                        tmem_wait_ld<U>(w);
                    }
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        const int row = m.r0 + s0 + u;
                        if (col && row < m.r1) {
                            S zv[W];
                            if (z_tm)
                                from_words<W>(w[u], zv);
                            else
                                VecIO<S, W>::load(z + ((size_t)(ya + row) * ne + x0), zv);
                            g_chunk<W>(gamma, zv, sp + (size_t)(row + 2) * ne + x0);
                        }
                    }
                }
            }
            __syncthreads();
            AT a = AT(0);
            s_march01<true>(a);
            acc[0] = a;
            acc[1] = AT(0);
        } else {
            acc[0] = acc[1] = AT(0);
        }
    }
    template <int W>
    __device__ static void g_chunk(C gamma, const S (&zv)[W], float *pp)
    {
        using A2 = typename InnerAr<PREC>::T;
        float4 *d4 = reinterpret_cast<float4 *>(pp);
#pragma unroll
        for (int v = 0; v < W; v += 4) {
            float4 t;
            round_pair<PREC>(A2::mul(gamma, PT::ld(zv[v])), A2::mul(gamma, PT::ld(zv[v + 1])), t.x, t.y);
            round_pair<PREC>(A2::mul(gamma, PT::ld(zv[v + 2])), A2::mul(gamma, PT::ld(zv[v + 3])), t.z, t.w);
            d4[v / 4] = t;
        }
    }
    // s1: p = fl_s(t + beta p_old) (p = t at j = 0) on the slab, then
    // acc = u.u with u = fl_s(S p) on the own rows
    __device__ GADI_RES_FN void s1_tm(int j, C beta, AT (&acc)[2]) const
    {
        if constexpr (TM_OK) {
            constexpr int W = WI, U = 4;
            int ya, yb;
            res_rows(ya, yb);
            const int R = yb - ya, nxw = ne / W;
            float *sp = res_smem();
            const S *t = (const S *)P.r;
            const bool first = j == 0;
            // halo rows -2, -1, R, R + 1 inside the grid: the neighbours' t
            const int nh = 4 * nxw;
            for (int i0 = threadIdx.x; i0 < nh; i0 += U * (int)blockDim.x) {
                S tv[U][W];
                int rowu[U], cu[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int i = i0 + u * (int)blockDim.x;
                    rowu[u] = -100;
                    if (i < nh) {
                        const int k = i / nxw, c = i - k * nxw, row = k < 2 ? k - 2 : R + k - 2;
                        if (ya + row >= 0 && ya + row < ny) {
                            rowu[u] = row;
                            cu[u] = c;
                            VecIO<S, W>::load(t + ((long long)(ya + row) * ne + (long long)c * W), tv[u]);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < U; u++)
                    if (rowu[u] != -100)
                        p_chunk<W>(first, beta, tv[u], sp + (size_t)(rowu[u] + 2) * ne + (size_t)cu[u] * W);
            }
            // own rows: t from TMEM
            const ResMap m = res_map(R, nxw);
            for (int cp = 0; cp < m.ncp; ++cp) {
                const int cx = m.cx0 + cp * (int)blockDim.x;
                const bool col = m.act && cx < nxw;
                const int x0 = col ? cx * W : 0;
                const int sb = cp * m.rmax;
                for (int s0 = 0; s0 < m.rmax; s0 += U) {
                    unsigned w[U][4];
#pragma unroll
                    for (int u = 0; u < U; u++) w[u][0] = w[u][1] = w[u][2] = w[u][3] = 0u;
#pragma unroll
                    for (int u = 0; u < U; u++)
                        if (s0 + u < m.rmax) tmem_ld4(tm_addr(sb + s0 + u, 1), w[u]);
                    tmem_wait_ld<U>(w);
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        const int row = m.r0 + s0 + u;
                        if (col && row < m.r1) {
                            S tv[W];
                            from_words<W>(w[u], tv);
                            p_chunk<W>(first, beta, tv, sp + (size_t)(row + 2) * ne + x0);
                        }
                    }
                }
            }
            __syncthreads();
            AT a = AT(0);
            s_march01<false>(a);
            acc[0] = a;
            acc[1] = AT(0);
        } else {
            acc[0] = acc[1] = AT(0);
        }
    }
    // the column march of s0 (T_OUT: t = fl_s(S^T g) to TMEM and the edge
    // rows to global memory, acc = t.t) and of s1 (acc = u.u, u = fl_s(S p))
    template <bool T_OUT>
    __device__ void s_march01(AT &acc) const
    {
        constexpr int W = WI;
        using A2 = typename InnerAr<PREC>::T;
        int ya, yb;
        res_rows(ya, yb);
        const int R = yb - ya, nxw = ne / W;
        const float *sp = res_smem();
        const ResMap m = res_map(R, nxw);
        const int lane = threadIdx.x & 31;
        const Coef7<C> &cf = T_OUT ? ct : cs;
        for (int cp = 0; cp < m.ncp; ++cp) {
            const int cx = m.cx0 + cp * (int)blockDim.x;
            const bool col = m.act && cx < nxw;
            const int x0 = col ? cx * W : 0;
            const bool lsh = lane > 0 && cx > 0, rsh = lane < 31 && cx + 1 < nxw;
            const bool xlo = x0 > 0, xhi = x0 + W < ne;
            // the slab row above the current one (slot = row + 2)
            const float *up_p = sp + (size_t)(m.r0 + 3) * ne + x0;
            S *tg = (S *)P.r + ((size_t)(ya + m.r0) * ne + x0);
            const int sb = cp * m.rmax;
            float dn[W], c[W], up[W];
#pragma unroll
            for (int v = 0; v < W; v++) dn[v] = c[v] = up[v] = 0.f;
            if (col) {
                res_row<W>(up_p - 2 * (size_t)ne, dn);
                res_row<W>(up_p - (size_t)ne, c);
            }
            int left = col ? m.r1 - m.r0 : 0;
            for (int st = 0; st < m.rmax; ++st) {
                const bool ok = left > 0;
                if (ok) res_row<W>(up_p, up);
                float cl = __shfl_up_sync(0xffffffffu, c[W - 1], 1);
                float cr = __shfl_down_sync(0xffffffffu, c[0], 1);
                S o[W];
#pragma unroll
                for (int v = 0; v < W; v++) o[v] = PT::st(C(0));
                if (ok) {
                    if (!lsh) cl = xlo ? up_p[-(ptrdiff_t)ne - 1] : 0.f;
                    if (!rsh) cr = xhi ? up_p[-(ptrdiff_t)ne + W] : 0.f;
#pragma unroll
                    for (int v = 0; v < W; v++) {
                        const float wv = v > 0 ? c[v - 1] : cl, ev = v + 1 < W ? c[v + 1] : cr;
                        o[v] = PT::st(stencil_at<A2, C, false, false>(cf.d, cf.c, C(0), c[v], wv, ev, dn[v], up[v],
                                                                      C(0), C(0), C(0), false));
                        const C q = PT::ld(o[v]);
                        acc += (AT)q * (AT)q;
                    }
                    if constexpr (T_OUT) {
                        if (s_edge(m.r0 + st, R, ya, yb)) VecIO<S, W>::store(tg, o);
                    }
                }
                if constexpr (T_OUT) {
                    unsigned w4[4];
                    to_words<W>(o, w4);
                    tmem_st4(tm_addr(sb + st, 1), w4);
                }
                --left;
                up_p += ne;
                tg += ne;
#pragma unroll
                for (int v = 0; v < W; v++) {
                    dn[v] = c[v];
                    c[v] = up[v];
                }
            }
        }
        if constexpr (T_OUT) tmem_wait_st();
    }
    // u = fl_s(S p) at one chunk of slab row k from p rows k - 1, k, k + 1
    // (lo, mid, hi) and the west / east neighbours of mid; zero outside the
    // grid's rows
    template <int W>
    __device__ void u_chunk(const float (&lo)[W], const float (&mid)[W], const float (&hi)[W], float ml, float mr,
                            bool inside, float (&u)[W]) const
    {
        using A2 = typename InnerAr<PREC>::T;
#pragma unroll
        for (int v = 0; v < W; v++) {
            const float wv = v > 0 ? mid[v - 1] : ml, ev = v + 1 < W ? mid[v + 1] : mr;
            u[v] = inside ? PT::ld(PT::st(stencil_at<A2, C, false, false>(cs.d, cs.c, C(0), mid[v], wv, ev, lo[v],
                                                                           hi[v], C(0), C(0), C(0), false)))
                          : 0.f;
        }
    }
    // u = fl_s(S p) at the single element x of slab row k (p read from the
    // slab; zero outside the grid)
    __device__ float u_point(const float *sp, int k, int x, bool inside) const
    {
        using A2 = typename InnerAr<PREC>::T;
        if (!inside || x < 0 || x >= ne) return 0.f;
        const float *r = sp + (size_t)(k + 2) * ne;
        const float pw = x > 0 ? r[x - 1] : 0.f, pe = x + 1 < ne ? r[x + 1] : 0.f;
        return PT::ld(PT::st(stencil_at<A2, C, false, false>(cs.d, cs.c, C(0), r[x], pw, pe, r[x - (ptrdiff_t)ne],
                                                             r[x + ne], C(0), C(0), C(0), false)));
    }
    // s2: y = fl_s(y + a p) (a p at j = 0), t = fl_s(t - a S^T u) with
    // u = fl_s(S p) recomputed, acc = t.t; t of the edge rows to global
    __device__ GADI_RES_FN void s2_tm(bool first, C a_, AT (&acc)[2]) const
    {
        if constexpr (TM_OK) {
            constexpr int W = WI;
            using A2 = typename InnerAr<PREC>::T;
            int ya, yb;
            res_rows(ya, yb);
            const int R = yb - ya, nxw = ne / W;
            const float *sp = res_smem();
            const ResMap m = res_map(R, nxw);
            const int lane = threadIdx.x & 31;
            AT s2 = AT(0);
            for (int cp = 0; cp < m.ncp; ++cp) {
                const int cx = m.cx0 + cp * (int)blockDim.x;
                const bool col = m.act && cx < nxw;
                const int x0 = col ? cx * W : 0;
                const bool lsh = lane > 0 && cx > 0, rsh = lane < 31 && cx + 1 < nxw;
                const bool xlo = x0 > 0, xhi = x0 + W < ne;
                // slab row pointer of p at row k: sp + (k + 2) ne + x0
                const float *pk = sp + (size_t)(m.r0 + 2) * ne + x0; // row r0
                S *tg = (S *)P.r + ((size_t)(ya + m.r0) * ne + x0);
                const int sb = cp * m.rmax;
                unsigned w[2][4]; // y, t of the current step
#pragma unroll
                for (int k = 0; k < 2; k++) w[k][0] = w[k][1] = w[k][2] = w[k][3] = 0u;
                if (!first) tmem_ld4(tm_addr(sb, 0), w[0]);
                tmem_ld4(tm_addr(sb, 1), w[1]);
                // p rows i - 1, i, i + 1 and u rows i - 1, i (i = r0)
                float pa[W], pb[W], pc[W], ua[W], ub[W];
#pragma unroll
                for (int v = 0; v < W; v++) pa[v] = pb[v] = pc[v] = ua[v] = ub[v] = 0.f;
                {
                    float pz[W]; // p row r0 - 2
#pragma unroll
                    for (int v = 0; v < W; v++) pz[v] = 0.f;
                    if (col) {
                        res_row<W>(pk - 2 * (size_t)ne, pz);
                        res_row<W>(pk - (size_t)ne, pa);
                        res_row<W>(pk, pb);
                        res_row<W>(pk + ne, pc);
                    }
                    // u(r0 - 1) from p(r0 - 2), p(r0 - 1), p(r0)
                    float ml = __shfl_up_sync(0xffffffffu, pa[W - 1], 1);
                    float mr = __shfl_down_sync(0xffffffffu, pa[0], 1);
                    if (col) {
                        if (!lsh) ml = xlo ? pk[-(ptrdiff_t)ne - 1] : 0.f;
                        if (!rsh) mr = xhi ? pk[-(ptrdiff_t)ne + W] : 0.f;
                    }
                    u_chunk<W>(pz, pa, pb, ml, mr, col && ya + m.r0 - 1 >= 0, ua);
                    // u(r0) from p(r0 - 1), p(r0), p(r0 + 1)
                    ml = __shfl_up_sync(0xffffffffu, pb[W - 1], 1);
                    mr = __shfl_down_sync(0xffffffffu, pb[0], 1);
                    if (col) {
                        if (!lsh) ml = xlo ? pk[-1] : 0.f;
                        if (!rsh) mr = xhi ? pk[W] : 0.f;
                    }
                    u_chunk<W>(pa, pb, pc, ml, mr, col, ub);
                }
                int left = col ? m.r1 - m.r0 : 0;
                for (int st = 0; st < m.rmax; ++st) {
                    const bool ok = left > 0;
                    const int row = m.r0 + st; // i
                    // p(i + 2), then u(i + 1) from p(i), p(i + 1), p(i + 2)
                    float pd[W], uc[W];
#pragma unroll
                    for (int v = 0; v < W; v++) pd[v] = 0.f;
                    if (ok) res_row<W>(pk + 2 * (size_t)ne, pd);
                    float ml = __shfl_up_sync(0xffffffffu, pc[W - 1], 1);
                    float mr = __shfl_down_sync(0xffffffffu, pc[0], 1);
                    if (ok) {
                        if (!lsh) ml = xlo ? pk[(ptrdiff_t)ne - 1] : 0.f;
                        if (!rsh) mr = xhi ? pk[(ptrdiff_t)ne + W] : 0.f;
                    }
                    u_chunk<W>(pb, pc, pd, ml, mr, ok && ya + row + 1 < ny, uc);
                    // S^T u at row i: west / east u(i) from the adjacent lanes,
                    // else recomputed from the slab
                    float ul = __shfl_up_sync(0xffffffffu, ub[W - 1], 1);
                    float ur = __shfl_down_sync(0xffffffffu, ub[0], 1);
                    C q[W];
#pragma unroll
                    for (int v = 0; v < W; v++) q[v] = C(0);
                    if (ok) {
                        if (!lsh) ul = xlo ? u_point(sp, row, x0 - 1, true) : 0.f;
                        if (!rsh) ur = xhi ? u_point(sp, row, x0 + W, true) : 0.f;
#pragma unroll
                        for (int v = 0; v < W; v++) {
                            const float wv = v > 0 ? ub[v - 1] : ul, ev = v + 1 < W ? ub[v + 1] : ur;
                            q[v] = stencil_at<A2, C, false, false>(ct.d, ct.c, C(0), ub[v], wv, ev, ua[v], uc[v], C(0),
                                                                  C(0), C(0), false);
                        }
                    }
                    tmem_wait_ld<2>(w);
                    S yv[W], tv[W];
                    from_words<W>(w[0], yv);
                    from_words<W>(w[1], tv);
                    if (ok) {
#pragma unroll
                        for (int v = 0; v < W; v++) {
                            yv[v] = PT::st(first ? A2::mul(a_, pb[v]) : A2::madd(a_, pb[v], PT::ld(yv[v])));
                            tv[v] = PT::st(A2::madd(-a_, q[v], PT::ld(tv[v])));
                            const C t2 = PT::ld(tv[v]);
                            s2 += (AT)t2 * (AT)t2;
                        }
                        if (s_edge(row, R, ya, yb)) VecIO<S, W>::store(tg, tv);
                    }
                    to_words<W>(yv, w[0]);
                    to_words<W>(tv, w[1]);
                    tmem_st4(tm_addr(sb + st, 0), w[0]);
                    tmem_st4(tm_addr(sb + st, 1), w[1]);
                    if (st + 1 < m.rmax) {
                        if (!first) tmem_ld4(tm_addr(sb + st + 1, 0), w[0]);
                        tmem_ld4(tm_addr(sb + st + 1, 1), w[1]);
                    }
                    --left;
                    pk += ne;
                    tg += ne;
#pragma unroll
                    for (int v = 0; v < W; v++) {
                        pa[v] = pb[v];
                        pb[v] = pc[v];
                        pc[v] = pd[v];
                        ua[v] = ub[v];
                        ub[v] = uc[v];
                    }
                }
            }
            tmem_wait_st();
            acc[0] = s2;
            acc[1] = AT(0);
        } else {
            acc[0] = acc[1] = AT(0);
        }
    }
    __device__ void s_flush_tm() const { tm_flush(0, (S *)P.y, 0); }

    // complex class: S = alpha I + i T (T = sigma I or diag(T_i)),
    // y = fl_s(g / (alpha + i T_i)) pointwise
    __device__ void s_pointwise(C gamma) const
    {
        if constexpr (K == 2) {
            using AE = ArExact<C>;
            const C ar = cs.d;
            const C den0 = AE::add(AE::mul(ar, ar), AE::mul(cs.e, cs.e));
            const S *z = (const S *)P.z;
            S *y = (S *)P.y;
            const long long np = (long long)P.nx * ny;
            for (long long i = vg.tid(); i < np; i += vg.nthreads()) {
                // a per-point T_i is rounded to u_s, as a stored coefficient
                const C ai = P.sig ? PT::ld(PT::from_f64(__ldg(P.sig + i))) : cs.e;
                const C den = P.sig ? AE::add(AE::mul(ar, ar), AE::mul(ai, ai)) : den0;
                const C gr = PT::ld(PT::st(A::mul(gamma, PT::ld(z[2 * i]))));
                const C gi = PT::ld(PT::st(A::mul(gamma, PT::ld(z[2 * i + 1]))));
                const C yr = AE::div(AE::add(AE::mul(gr, ar), AE::mul(gi, ai)), den);
                const C yi = AE::div(AE::add(AE::mul(gi, ar), -AE::mul(gr, ai)), den);
                y[2 * i] = PT::st(yr);
                y[2 * i + 1] = PT::st(yi);
            }
        }
    }
};

} // namespace gadi
