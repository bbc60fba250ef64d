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

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// arithmetic policies
// ---------------------------------------------------------------------------
// Exact: every product and sum rounded separately, in the operation order of
// the method's definition (no contraction into FMA).  Used for FP32/BF16
// arithmetic and for the FP64 residual / operator application.
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
// Fused: products folded into FMA.  Used for the all-FP64 inner solves, where
// the FP64 pipe, not memory, is the scarcer resource on this GPU.
struct ArFusedD {
    __device__ static double mul(double a, double b) { return a * b; }
    __device__ static double add(double a, double b) { return a + b; }
    __device__ static double madd(double a, double b, double s) { return fma(a, b, s); }
    __device__ static double div(double a, double b) { return a / b; }
};
template <int PREC> struct InnerAr { using T = ArExact<float>; };
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

template <class C> struct Coef7 {
    C d, c[6], e;
};

// ---------------------------------------------------------------------------
// the marching sweep over a 2D or 3D grid
// ---------------------------------------------------------------------------
// A warp owns a strip of 32*W consecutive elements of a row (W per lane) and
// marches along the slowest axis (y in 2D, z in 3D) over a contiguous range
// of its work units, keeping the field at m-1, m, m+1 in registers.  x
// neighbours come from warp shuffles (lane 0 / 31 evaluate the field one
// element past the strip); 3D y neighbours are evaluated directly.  The field
// is zero outside the grid (Dirichlet).  Work units are split evenly and
// contiguously over all warps of the grid.
// field values of W consecutive elements at g, or zeros when `valid` is false
template <int W, class Ph>
__device__ __forceinline__ void load_row(const Ph &ph, bool valid, long long g, typename Ph::FT (&o)[W])
{
    if (valid) {
        ph.fv(g, o);
    } else {
#pragma unroll
        for (int v = 0; v < W; v++) o[v] = typename Ph::FT(0);
    }
}

template <int W, int K, bool D3, class Ph, class AT>
__device__ __forceinline__ void march(const Ph &ph, int ne, int ny, int nz, AT (&acc)[2])
{
    using FT = typename Ph::FT;
    const int lane = threadIdx.x & 31;
    const int nstrips = (ne + 32 * W - 1) / (32 * W);
    const int collen = D3 ? nz : ny;
    const long long ncols = D3 ? (long long)nstrips * ny : (long long)nstrips;
    const long long mstride = D3 ? (long long)ne * ny : (long long)ne;
    const long long nunits = ncols * collen;
    const long long GW = (long long)gridDim.x * (blockDim.x >> 5);
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    long long u = nunits * gw / GW;
    const long long u1 = nunits * (gw + 1) / GW;
    while (u < u1) {
        const long long col = u / collen;
        const int m0 = (int)(u - col * collen);
        const int m1 = (int)min((long long)collen, (long long)m0 + (u1 - u));
        u += m1 - m0;
        const int strip = D3 ? (int)(col / ny) : (int)col;
        const int yy = D3 ? (int)(col - (long long)strip * ny) : 0;
        const int e0 = strip * 32 * W + lane * W;
        const bool act = e0 < ne;
        const long long cbase = (D3 ? (long long)yy * ne : 0ll) + e0;
        FT dn[W], cu[W], up[W];
        load_row<W>(ph, act && m0 - 1 >= 0, cbase + (long long)(m0 - 1) * mstride, dn);
        load_row<W>(ph, act, cbase + (long long)m0 * mstride, cu);
        for (int m = m0; m < m1; ++m) {
            load_row<W>(ph, act && m + 1 < collen, cbase + (long long)(m + 1) * mstride, up);
            const long long g = cbase + (long long)m * mstride;
            FT lh[K], rh[K];
#pragma unroll
            for (int k = 0; k < K; k++) {
                lh[k] = __shfl_up_sync(0xffffffffu, cu[W - K + k], 1);
                rh[k] = __shfl_down_sync(0xffffffffu, cu[k], 1);
            }
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < K; k++) lh[k] = (act && e0 > 0) ? ph.f1(g - K + k) : FT(0);
            }
            if (lane == 31) {
#pragma unroll
                for (int k = 0; k < K; k++) rh[k] = (act && e0 + W < ne) ? ph.f1(g + W + k) : FT(0);
            }
            FT w[W], e[W];
#pragma unroll
            for (int v = 0; v < W; v++) {
                w[v] = (v >= K) ? cu[v - K] : lh[v];
                e[v] = (v + K < W) ? cu[v + K] : rh[v + K - W];
            }
            if (act) {
                if constexpr (D3) {
                    FT sy[W], ny_[W];
                    load_row<W>(ph, yy > 0, g - ne, sy);
                    load_row<W>(ph, yy + 1 < ny, g + ne, ny_);
                    ph.out(g, cu, w, e, sy, ny_, dn, up, acc);
                } else {
                    ph.out(g, cu, w, e, dn, up, dn, up, acc);
                }
            }
#pragma unroll
            for (int v = 0; v < W; v++) {
                dn[v] = cu[v];
                cu[v] = up[v];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// stencil phases
// ---------------------------------------------------------------------------
template <int PREC, int W, int K, bool D3>
struct PhResidual { // R (and MODE_APPLY with b == nullptr, y == nullptr)
    using PT = Prec<PREC>;
    using S = typename PT::S;
    using FT = double;
    using A = ArExact<double>;
    const double *x;
    const S *y;
    double *xo;
    const double *b;
    double *rout;
    S *rs;
    Coef7<double> cf;
    __device__ double f1(long long g) const
    {
        double v = __ldcg(x + g);
        if (y) v = A::add(v, PT::to_f64(y[g]));
        return v;
    }
    __device__ void fv(long long g, double (&o)[W]) const
    {
        VecIO<double, W>::load(x + g, o);
        if (y) {
            S yv[W];
            VecIO<S, W>::load(y + g, yv);
#pragma unroll
            for (int v = 0; v < W; v++) o[v] = A::add(o[v], PT::to_f64(yv[v]));
        }
    }
    __device__ void out(long long g, const double (&c)[W], const double (&w)[W], const double (&e)[W],
                        const double (&s)[W], const double (&n)[W], const double (&bb)[W],
                        const double (&t)[W], double (&acc)[2]) const
    {
        double ax[W];
#pragma unroll
        for (int v = 0; v < W; v++)
            ax[v] = stencil_at<A, double, D3, K == 2>(cf.d, cf.c, cf.e, c[v], w[v], e[v], s[v], n[v],
                                                      bb[v], t[v], c[v ^ (K - 1)], (v & 1) != 0);
        if (b == nullptr) { // operator application: xo = Op x
            VecIO<double, W>::store(xo + g, ax);
            return;
        }
        double bv[W], r[W];
        S so[W];
        VecIO<double, W>::load(b + g, bv);
#pragma unroll
        for (int v = 0; v < W; v++) {
            r[v] = __dsub_rn(bv[v], ax[v]);
            acc[0] = fma(r[v], r[v], acc[0]);
            so[v] = PT::from_f64(r[v]);
            const double sv = PT::to_f64(so[v]);
            acc[1] = fma(sv, sv, acc[1]);
        }
        VecIO<double, W>::store(xo + g, c);
        VecIO<S, W>::store(rs + g, so);
        if (rout) VecIO<double, W>::store(rout + g, r);
    }
};

// p = fl_s(src + beta p_old) as a field (src = r for H1, t for S1)
template <int PREC, int W>
struct FieldDir {
    using PT = Prec<PREC>;
    using S = typename PT::S;
    using C = typename PT::C;
    using A = typename InnerAr<PREC>::T;
    const S *src, *pold;
    C beta;
    bool first;
    __device__ C f1(long long g) const
    {
        C v = PT::ld(src[g]);
        if (!first) v = A::madd(beta, PT::ld(pold[g]), v);
        return PT::ld(PT::st(v));
    }
    __device__ void fv(long long g, C (&o)[W]) const
    {
        S sv[W];
        VecIO<S, W>::load(src + g, sv);
        if (first) {
#pragma unroll
            for (int v = 0; v < W; v++) o[v] = PT::ld(sv[v]);
        } else {
            S pv[W];
            VecIO<S, W>::load(pold + g, pv);
#pragma unroll
            for (int v = 0; v < W; v++) o[v] = PT::ld(PT::st(A::madd(beta, PT::ld(pv[v]), PT::ld(sv[v]))));
        }
    }
};

// plain u_s field, optionally scaled and re-rounded: fl_s(scale * v)
template <int PREC, int W, bool SCALE>
struct FieldLoad {
    using PT = Prec<PREC>;
    using S = typename PT::S;
    using C = typename PT::C;
    using A = typename InnerAr<PREC>::T;
    const S *src;
    C scale;
    __device__ C f1(long long g) const
    {
        if constexpr (SCALE) return PT::ld(PT::st(A::mul(scale, PT::ld(src[g]))));
        else return PT::ld(src[g]);
    }
    __device__ void fv(long long g, C (&o)[W]) const
    {
        S sv[W];
        VecIO<S, W>::load(src + g, sv);
#pragma unroll
        for (int v = 0; v < W; v++) {
            if constexpr (SCALE) o[v] = PT::ld(PT::st(A::mul(scale, PT::ld(sv[v]))));
            else o[v] = PT::ld(sv[v]);
        }
    }
};

template <int PREC, int W, int K, bool D3>
struct PhH1 : FieldDir<PREC, W> { // p = fl_s(r + beta p_old); sum p.(H p)
    using Base = FieldDir<PREC, W>;
    using C = typename Base::C;
    using S = typename Base::S;
    using PT = Prec<PREC>;
    using FT = C;
    using AT = typename AccT<PREC>::T;
    S *pnew;
    Coef7<C> h;
    __device__ void out(long long g, const C (&c)[W], const C (&w)[W], const C (&e)[W], const C (&s)[W],
                        const C (&n)[W], const C (&b)[W], const C (&t)[W], AT (&acc)[2]) const
    {
        S ps[W];
#pragma unroll
        for (int v = 0; v < W; v++) {
            const C q = stencil_at<typename Base::A, C, D3, false>(h.d, h.c, C(0), c[v], w[v], e[v], s[v],
                                                                  n[v], b[v], t[v], C(0), false);
            acc[0] += (AT)c[v] * (AT)q;
            ps[v] = PT::st(c[v]);
        }
        VecIO<S, W>::store(pnew + g, ps);
    }
};

template <int PREC, int W, int K, bool D3>
struct PhH2 : FieldLoad<PREC, W, false> { // z += a p, r -= a H p; sum r.r
    using Base = FieldLoad<PREC, W, false>;
    using C = typename Base::C;
    using S = typename Base::S;
    using PT = Prec<PREC>;
    using FT = C;
    using AT = typename AccT<PREC>::T;
    using A = typename Base::A;
    S *z, *r;
    C a;
    bool first;
    Coef7<C> h;
    __device__ void out(long long g, const C (&c)[W], const C (&w)[W], const C (&e)[W], const C (&s)[W],
                        const C (&n)[W], const C (&b)[W], const C (&t)[W], AT (&acc)[2]) const
    {
        S zv[W], rv[W];
        if (!first) VecIO<S, W>::load(z + g, zv);
        VecIO<S, W>::load(r + g, rv);
#pragma unroll
        for (int v = 0; v < W; v++) {
            const C q = stencil_at<A, C, D3, false>(h.d, h.c, C(0), c[v], w[v], e[v], s[v], n[v], b[v],
                                                    t[v], C(0), false);
            const C zn = first ? A::mul(a, c[v]) : A::madd(a, c[v], PT::ld(zv[v]));
            zv[v] = PT::st(zn);
            rv[v] = PT::st(A::madd(-a, q, PT::ld(rv[v])));
            const C rr = PT::ld(rv[v]);
            acc[0] += (AT)rr * (AT)rr;
        }
        VecIO<S, W>::store(z + g, zv);
        VecIO<S, W>::store(r + g, rv);
    }
};

template <int PREC, int W, int K, bool D3>
struct PhS0 : FieldLoad<PREC, W, true> { // t = fl_s(S^T fl_s(gamma z)); sum t.t
    using Base = FieldLoad<PREC, W, true>;
    using C = typename Base::C;
    using S = typename Base::S;
    using PT = Prec<PREC>;
    using FT = C;
    using AT = typename AccT<PREC>::T;
    using A = typename Base::A;
    S *t;
    Coef7<C> st;
    __device__ void out(long long g, const C (&c)[W], const C (&w)[W], const C (&e)[W], const C (&s)[W],
                        const C (&n)[W], const C (&b)[W], const C (&tt)[W], AT (&acc)[2]) const
    {
        S to[W];
#pragma unroll
        for (int v = 0; v < W; v++) {
            const C q = stencil_at<A, C, D3, K == 2>(st.d, st.c, st.e, c[v], w[v], e[v], s[v], n[v], b[v],
                                                     tt[v], c[v ^ (K - 1)], (v & 1) != 0);
            to[v] = PT::st(q);
            const C qq = PT::ld(to[v]);
            acc[0] += (AT)qq * (AT)qq;
        }
        VecIO<S, W>::store(t + g, to);
    }
};

template <int PREC, int W, int K, bool D3>
struct PhS1 : FieldDir<PREC, W> { // p = fl_s(t + beta p_old), u = fl_s(S p); sum u.u
    using Base = FieldDir<PREC, W>;
    using C = typename Base::C;
    using S = typename Base::S;
    using PT = Prec<PREC>;
    using FT = C;
    using AT = typename AccT<PREC>::T;
    S *pnew, *u;
    Coef7<C> sc;
    __device__ void out(long long g, const C (&c)[W], const C (&w)[W], const C (&e)[W], const C (&s)[W],
                        const C (&n)[W], const C (&b)[W], const C (&t)[W], AT (&acc)[2]) const
    {
        S ps[W], us[W];
#pragma unroll
        for (int v = 0; v < W; v++) {
            const C q = stencil_at<typename Base::A, C, D3, K == 2>(sc.d, sc.c, sc.e, c[v], w[v], e[v], s[v],
                                                                   n[v], b[v], t[v], c[v ^ (K - 1)],
                                                                   (v & 1) != 0);
            us[v] = PT::st(q);
            const C uu = PT::ld(us[v]);
            acc[0] += (AT)uu * (AT)uu;
            ps[v] = PT::st(c[v]);
        }
        VecIO<S, W>::store(pnew + g, ps);
        VecIO<S, W>::store(u + g, us);
    }
};

template <int PREC, int W, int K, bool D3>
struct PhS2 : FieldLoad<PREC, W, false> { // y += a p, t -= a S^T u; sum t.t
    using Base = FieldLoad<PREC, W, false>;
    using C = typename Base::C;
    using S = typename Base::S;
    using PT = Prec<PREC>;
    using FT = C;
    using AT = typename AccT<PREC>::T;
    using A = typename Base::A;
    const S *p;
    S *y, *t;
    C a;
    bool first;
    Coef7<C> st;
    __device__ void out(long long g, const C (&c)[W], const C (&w)[W], const C (&e)[W], const C (&s)[W],
                        const C (&n)[W], const C (&b)[W], const C (&tt)[W], AT (&acc)[2]) const
    {
        S pv[W], yv[W], tv[W];
        VecIO<S, W>::load(p + g, pv);
        if (!first) VecIO<S, W>::load(y + g, yv);
        VecIO<S, W>::load(t + g, tv);
#pragma unroll
        for (int v = 0; v < W; v++) {
            const C q = stencil_at<A, C, D3, K == 2>(st.d, st.c, st.e, c[v], w[v], e[v], s[v], n[v], b[v],
                                                     tt[v], c[v ^ (K - 1)], (v & 1) != 0);
            const C pp = PT::ld(pv[v]);
            yv[v] = PT::st(first ? A::mul(a, pp) : A::madd(a, pp, PT::ld(yv[v])));
            tv[v] = PT::st(A::madd(-a, q, PT::ld(tv[v])));
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
template <int KIND, int PREC, int WI, int WR>
struct StencilImpl {
    using PT = Prec<PREC>;
    using S = typename PT::S;
    using C = typename PT::C;
    using A = typename InnerAr<PREC>::T;
    using AT = typename AccT<PREC>::T;
    static constexpr int K = (KIND == K_C2D5) ? 2 : 1;
    static constexpr bool D3 = (KIND == K_3D7);
    const Params &P;
    int ne, ny, nz;
    Coef7<double> ca;
    Coef7<C> ch, cs, ct;

    __device__ explicit StencilImpl(const Params &p) : P(p)
    {
        ne = p.nx * K;
        ny = p.ny;
        nz = D3 ? p.nz : 1;
        ca.d = p.co.a_d; ca.e = p.co.a_e;
        ch.d = (C)p.co.h_d; ch.e = C(0);
        cs.d = (C)p.co.s_d; cs.e = (C)p.co.s_e;
        ct.d = (C)p.co.t_d; ct.e = (C)p.co.t_e;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            ca.c[k] = p.co.a_c[k];
            ch.c[k] = (C)p.co.h_c[k];
            cs.c[k] = (C)p.co.s_c[k];
            ct.c[k] = (C)p.co.t_c[k];
        }
    }

    __device__ void residual(const double *xin, const S *y, double *xout, double (&acc)[2]) const
    {
        PhResidual<PREC, WR, K, D3> ph{xin, y, xout, P.b, P.r_out, (S *)P.r, ca};
        double a[2] = {0.0, 0.0};
        march<WR, K, D3>(ph, ne, ny, nz, a);
        acc[0] = a[0];
        acc[1] = a[1];
    }
    __device__ void apply(const double *x, double *yout) const
    {
        PhResidual<PREC, WR, K, D3> ph{x, nullptr, yout, nullptr, nullptr, nullptr, ca};
        double a[2] = {0.0, 0.0};
        march<WR, K, D3>(ph, ne, ny, nz, a);
    }
    __device__ void h1(bool first, C beta, const S *pold, S *pnew, double (&acc)[2]) const
    {
        PhH1<PREC, WI, K, D3> ph;
        ph.src = (const S *)P.r; ph.pold = pold; ph.beta = beta; ph.first = first;
        ph.pnew = pnew; ph.h = ch;
        AT a[2] = {AT(0), AT(0)};
        march<WI, K, D3>(ph, ne, ny, nz, a);
        acc[0] = (double)a[0];
        acc[1] = 0.0;
    }
    __device__ void h2(bool first, C a_, const S *p, double (&acc)[2]) const
    {
        PhH2<PREC, WI, K, D3> ph;
        ph.src = p; ph.scale = C(1); ph.z = (S *)P.z; ph.r = (S *)P.r; ph.a = a_; ph.first = first;
        ph.h = ch;
        AT a[2] = {AT(0), AT(0)};
        march<WI, K, D3>(ph, ne, ny, nz, a);
        acc[0] = (double)a[0];
        acc[1] = 0.0;
    }
    __device__ void s0(C gamma, double (&acc)[2]) const
    {
        PhS0<PREC, WI, K, D3> ph;
        ph.src = (const S *)P.z; ph.scale = gamma; ph.t = (S *)P.r; ph.st = ct;
        AT a[2] = {AT(0), AT(0)};
        march<WI, K, D3>(ph, ne, ny, nz, a);
        acc[0] = (double)a[0];
        acc[1] = 0.0;
    }
    __device__ void s1(bool first, C beta, const S *pold, S *pnew, double (&acc)[2]) const
    {
        PhS1<PREC, WI, K, D3> ph;
        ph.src = (const S *)P.r; ph.pold = pold; ph.beta = beta; ph.first = first;
        ph.pnew = pnew; ph.u = (S *)P.u; ph.sc = cs;
        AT a[2] = {AT(0), AT(0)};
        march<WI, K, D3>(ph, ne, ny, nz, a);
        acc[0] = (double)a[0];
        acc[1] = 0.0;
    }
    __device__ void s2(bool first, C a_, const S *p, double (&acc)[2]) const
    {
        PhS2<PREC, WI, K, D3> ph;
        ph.src = (const S *)P.u; ph.scale = C(1); ph.p = p; ph.y = (S *)P.y; ph.t = (S *)P.r;
        ph.a = a_; ph.first = first; ph.st = ct;
        AT a[2] = {AT(0), AT(0)};
        march<WI, K, D3>(ph, ne, ny, nz, a);
        acc[0] = (double)a[0];
        acc[1] = 0.0;
    }
    // complex class: S = (alpha + i sigma) I, y = fl_s(g / (alpha + i sigma))
    __device__ void s_pointwise(C gamma) const
    {
        if constexpr (K == 2) {
            using AE = ArExact<C>;
            const C ar = cs.d, ai = cs.e;
            const C den = AE::add(AE::mul(ar, ar), AE::mul(ai, ai));
            const S *z = (const S *)P.z;
            S *y = (S *)P.y;
            const long long np = (long long)P.nx * ny;
            for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np;
                 i += (long long)gridDim.x * blockDim.x) {
                const C gr = PT::ld(PT::st(A::mul(gamma, PT::ld(z[2 * i]))));
                const C gi = PT::ld(PT::st(A::mul(gamma, PT::ld(z[2 * i + 1]))));
                const C yr = AE::div(AE::add(AE::mul(gr, ar), AE::mul(gi, ai)), den);
                const C yi = AE::div(AE::add(AE::mul(gi, ar), -AE::mul(gr, ai)), den);
                y[2 * i] = PT::st(yr);
                y[2 * i + 1] = PT::st(yi);
            }
        }
    }
    __device__ bool csr_pre_sync() const { return false; }
};

} // namespace gadi
