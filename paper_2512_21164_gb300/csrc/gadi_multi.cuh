// Four right-hand sides of one 2D 5-point system interleaved: every vector of
// the solve stored as [n][4] (the four values of a grid point side by side),
// so a lane's 16-byte FP32 load holds one point of all four systems and one
// sweep, one barrier and one grid-wide sum serve all four.  Each right-hand
// side keeps its own CG and CGNR scalars, its own stopping decisions and its
// own outer iteration (Algorithm 1 for each); a right-hand side that has
// stopped is frozen (its step sizes are zero) while the others go on.
//
// The march of the single solve is reused with 4 elements per lane and an
// x-stride of 4 elements (the neighbours of element v of a point are element v
// of the points left and right), so element v of every vector is right-hand
// side v.  FP32 inner solves (u_s = FP32), FP64 residual and update.
#pragma once
#include "gadi_kernel.cuh"

namespace gadi {

constexpr int NR = 4; // right-hand sides per unit

// fl(src + beta_v p_old) with a step size per right-hand side (element v of
// a 4-aligned chunk is right-hand side v)
struct FieldDir4 {
    using PT = Prec<P_FP32>;
    using S = float;
    using C = float;
    using FT = float;
    using A = ArFusedF;
    const S *src, *pold;
    C beta[NR];
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
#pragma unroll
        for (int v = 0; v < N; v++) o[v] = first ? r.s[v] : A::madd(beta[v % NR], r.p[v], r.s[v]);
    }
};

// R (4 right-hand sides): x_out = x + y, r = b - A x_out in FP64 (the FP64
// stencil of the single solve, same order), r_s = fl(r); sums per right-hand
// side ||r||^2 (acc[v]) and ||r_s||^2 (acc[4 + v]) in FP64
struct PhResidual4 {
    using PT = Prec<P_FP32>;
    using S = float;
    using Fld = FieldX<P_FP32>;
    using Own = OwnIn<double, NR, 1>;
    Fld f;
    double *xo;
    const double *b;
    S *rs;
    Coef7<double> cf;
    __device__ void load_own(long long g, Own &o) const { VecIO<double, NR>::load(b + g, o.v[0]); }
    __device__ void out(long long g, const Own &o, const double (&c)[NR], const double (&w)[NR],
                        const double (&e)[NR], const double (&s)[NR], const double (&n)[NR], const double (&)[NR],
                        const double (&)[NR], double (&acc)[2 * NR]) const
    {
        double r[NR];
        S so[NR];
#pragma unroll
        for (int v = 0; v < NR; v++) {
            const double ax =
                stencil_at<ArFusedD, double, false, false>(cf.d, cf.c, 0.0, c[v], w[v], e[v], s[v], n[v], 0.0, 0.0, 0.0,
                                                           false);
            r[v] = __dsub_rn(o.v[0][v], ax);
            acc[v] = fma(r[v], r[v], acc[v]);
            so[v] = PT::from_f64(r[v]);
            const double d = f32_to_f64_fast(so[v]);
            acc[NR + v] = fma(d, d, acc[NR + v]);
        }
        VecIO<double, NR>::store(xo + g, c);
        VecIO<S, NR>::store(rs + g, so);
    }
};

// H1: p = fl(r + beta_v p_old); sums p.(H p) per right-hand side
struct PhH1_4 {
    using Fld = FieldDir4;
    using Own = OwnIn<float, NR, 0>;
    Fld f;
    float *pnew;
    Coef7<float> h;
    __device__ void load_own(long long, Own &) const {}
    __device__ void out(long long g, const Own &, const float (&c)[NR], const float (&w)[NR], const float (&e)[NR],
                        const float (&s)[NR], const float (&n)[NR], const float (&)[NR], const float (&)[NR],
                        float (&acc)[2 * NR]) const
    {
#pragma unroll
        for (int v = 0; v < NR; v++) {
            const float q = stencil_at<ArFusedF, float, false, false>(h.d, h.c, 0.f, c[v], w[v], e[v], s[v], n[v], 0.f,
                                                                      0.f, 0.f, false);
            acc[v] += c[v] * q;
        }
        VecIO<float, NR>::store(pnew + g, c);
    }
};

// H2: z = fl(z + a_v p), r = fl(r - a_v H p) with H p recomputed; sums r.r
struct PhH2_4 {
    using Fld = FieldLoad<P_FP32, false>;
    using Own = OwnIn<float, NR, 2>; // z, r
    Fld f;
    float *z, *r;
    float a[NR];
    bool first;
    Coef7<float> h;
    __device__ void load_own(long long g, Own &o) const
    {
        if (!first) VecIO<float, NR>::load(z + g, o.v[0]);
        VecIO<float, NR>::load(r + g, o.v[1]);
    }
    __device__ void out(long long g, const Own &o, const float (&c)[NR], const float (&w)[NR], const float (&e)[NR],
                        const float (&s)[NR], const float (&n)[NR], const float (&)[NR], const float (&)[NR],
                        float (&acc)[2 * NR]) const
    {
        float zv[NR], rv[NR];
#pragma unroll
        for (int v = 0; v < NR; v++) {
            const float q = stencil_at<ArFusedF, float, false, false>(h.d, h.c, 0.f, c[v], w[v], e[v], s[v], n[v], 0.f,
                                                                      0.f, 0.f, false);
            zv[v] = first ? __fmul_rn(a[v], c[v]) : __fmaf_rn(a[v], c[v], o.v[0][v]);
            rv[v] = __fmaf_rn(-a[v], q, o.v[1][v]);
            acc[v] += rv[v] * rv[v];
        }
        VecIO<float, NR>::store(z + g, zv);
        VecIO<float, NR>::store(r + g, rv);
    }
};

// S0: g = fl(gamma z) (the field), t = fl(S^T g); sums t.t
struct PhS0_4 {
    using Fld = FieldLoad<P_FP32, true>;
    using Own = OwnIn<float, NR, 0>;
    Fld f;
    float *t;
    Coef7<float> st;
    __device__ void load_own(long long, Own &) const {}
    __device__ void out(long long g, const Own &, const float (&c)[NR], const float (&w)[NR], const float (&e)[NR],
                        const float (&s)[NR], const float (&n)[NR], const float (&)[NR], const float (&)[NR],
                        float (&acc)[2 * NR]) const
    {
        float to[NR];
#pragma unroll
        for (int v = 0; v < NR; v++) {
            to[v] = stencil_at<ArFusedF, float, false, false>(st.d, st.c, 0.f, c[v], w[v], e[v], s[v], n[v], 0.f, 0.f,
                                                              0.f, false);
            acc[v] += to[v] * to[v];
        }
        VecIO<float, NR>::store(t + g, to);
    }
};

// S1: p = fl(t + beta_v p_old), u = fl(S p); sums u.u
struct PhS1_4 {
    using Fld = FieldDir4;
    using Own = OwnIn<float, NR, 0>;
    Fld f;
    float *pnew, *u;
    Coef7<float> sc;
    __device__ void load_own(long long, Own &) const {}
    __device__ void out(long long g, const Own &, const float (&c)[NR], const float (&w)[NR], const float (&e)[NR],
                        const float (&s)[NR], const float (&n)[NR], const float (&)[NR], const float (&)[NR],
                        float (&acc)[2 * NR]) const
    {
        float us[NR];
#pragma unroll
        for (int v = 0; v < NR; v++) {
            us[v] = stencil_at<ArFusedF, float, false, false>(sc.d, sc.c, 0.f, c[v], w[v], e[v], s[v], n[v], 0.f, 0.f,
                                                              0.f, false);
            acc[v] += us[v] * us[v];
        }
        VecIO<float, NR>::store(pnew + g, c);
        VecIO<float, NR>::store(u + g, us);
    }
};

// S2: y = fl(y + a_v p), t = fl(t - a_v S^T u); sums t.t
struct PhS2_4 {
    using Fld = FieldLoad<P_FP32, false>;
    using Own = OwnIn<float, NR, 3>; // p, y, t
    Fld f;
    const float *p;
    float *y, *t;
    float a[NR];
    bool first;
    Coef7<float> st;
    __device__ void load_own(long long g, Own &o) const
    {
        VecIO<float, NR>::load(p + g, o.v[0]);
        if (!first) VecIO<float, NR>::load(y + g, o.v[1]);
        VecIO<float, NR>::load(t + g, o.v[2]);
    }
    __device__ void out(long long g, const Own &o, const float (&c)[NR], const float (&w)[NR], const float (&e)[NR],
                        const float (&s)[NR], const float (&n)[NR], const float (&)[NR], const float (&)[NR],
                        float (&acc)[2 * NR]) const
    {
        float yv[NR], tv[NR];
#pragma unroll
        for (int v = 0; v < NR; v++) {
            const float q = stencil_at<ArFusedF, float, false, false>(st.d, st.c, 0.f, c[v], w[v], e[v], s[v], n[v], 0.f,
                                                                      0.f, 0.f, false);
            yv[v] = first ? __fmul_rn(a[v], o.v[0][v]) : __fmaf_rn(a[v], o.v[0][v], o.v[1][v]);
            tv[v] = __fmaf_rn(-a[v], q, o.v[2][v]);
            acc[v] += tv[v] * tv[v];
        }
        VecIO<float, NR>::store(y + g, yv);
        VecIO<float, NR>::store(t + g, tv);
    }
};

} // namespace gadi

namespace gadi {

// The four right-hand sides' scalars and decisions: one copy per block in
// shared memory.  Every thread of the group holds the same values (the
// grid-wide sums give every block the same totals); kept in registers they
// made the kernel spill.  Thread 0 updates them after each grid-wide sum, the
// block reads them after a block barrier.
struct State4 {
    double r0[NR], rel[NR];
    long long ih[NR], is[NR];
    int status[NR], kdone[NR], done[NR], act[NR], since[NR], its[NR];
    float rr[NR], best[NR], thr[NR], beta[NR], a[NR], rs2[NR];
    int any, all;
};

// Algorithm 1 for the four interleaved right-hand sides of a unit, on the
// group's blocks (VGrid vg).  Vectors: P.xm0 / P.xm1 (x, ping-pong), P.bm
// (b), P.r, P.z, P.p0, P.p1, P.y, P.u (u_s = FP32), all [n][4]; P.hist holds
// 4 x (P.maxit + 2) doubles (relres per outer iteration of each right-hand
// side); P.ctl points at 4 control blocks.  Returns false if a barrier gave up.
struct Runner4 {
    const Params &P;
    VGrid vg;
    GridSync gs;
    State4 &st;
    int slot = 0;
    int ne, ny;
    __device__ Runner4(const Params &p, VGrid g, State4 &s) : P(p), vg(g), st(s)
    {
        gs.counter = p.bar;
        gs.abort_flag = p.abort_flag;
        gs.nblocks = (unsigned)g.n;
        ne = p.nx * NR;
        ny = p.ny;
    }
    template <class RT> __device__ bool reduce(const RT (&acc)[2 * NR], RT (&out)[2 * NR])
    {
        const int G = vg.n;
        RT *part = reinterpret_cast<RT *>(P.part + (size_t)slot * 2 * NR * G);
        block_partials_write<2 * NR, RT>(acc, part, G, vg.b);
        if (!gs.sync()) return false;
        grid_partials_sum<2 * NR, RT>(part, G, out);
        slot ^= 1;
        return true;
    }
    template <class Ph, class RT> __device__ void sweep(const Ph &ph, RT (&acc)[2 * NR]) const
    {
#pragma unroll
        for (int k = 0; k < 2 * NR; k++) acc[k] = RT(0);
        march<NR, NR, false, 0>(ph, ne, ny, 1, acc, vg);
    }
    __device__ static bool t0() { return threadIdx.x == 0; }

    // thread 0: the stopping rules of an inner solve after a step with the
    // new residual norms `sum` (CG: r.r, CGNR: t.t); sets st.any
    __device__ void inner_update(int j, const float (&sum)[2 * NR]) const
    {
        int any = 0;
        for (int v = 0; v < NR; v++) {
            if (!st.act[v]) {
                st.beta[v] = 0.f;
                continue;
            }
            const float rn = sum[v];
            st.its[v] = j + 1;
            bool stop = rn <= st.thr[v] || !(rn == rn);
            if (!stop) {
                if (rn < st.best[v]) {
                    st.best[v] = rn;
                    st.since[v] = 0;
                } else if (P.inner_stag > 0 && ++st.since[v] >= P.inner_stag) {
                    stop = true;
                }
            }
            if (stop) {
                st.act[v] = 0;
                st.beta[v] = 0.f;
            } else {
                st.beta[v] = ArFusedF::div(rn, st.rr[v]);
                st.rr[v] = rn;
            }
            any |= st.act[v];
        }
        st.any = any;
    }
    // thread 0: start an inner solve for the right-hand sides still running
    // (st.done clear) from the initial norms rr0 and tolerance tol
    __device__ void inner_start(const float (&rr0)[NR], double tol) const
    {
        int any = 0;
        for (int v = 0; v < NR; v++) {
            st.its[v] = 0;
            st.rr[v] = st.best[v] = rr0[v];
            st.act[v] = !st.done[v] && rr0[v] > 0.f;
            st.thr[v] = floor_to<float>(tol * tol * (double)rr0[v]);
            st.beta[v] = 0.f;
            st.since[v] = 0;
            any |= st.act[v];
        }
        st.any = any;
    }

    // CG on H for the right-hand sides still running (norms ||r_s||^2 in
    // st.rs2); the others get z = 0.
    __device__ bool h_loop()
    {
        if (t0()) {
            float rr0[NR];
            for (int v = 0; v < NR; v++) rr0[v] = st.rs2[v];
            inner_start(rr0, P.tol_h);
        }
        __syncthreads();
        float acc[2 * NR], sum[2 * NR];
        for (int j = 0; j < P.maxit_inner; ++j) {
            float *pnew = (float *)((j & 1) ? P.p1 : P.p0);
            const float *pold = (const float *)((j & 1) ? P.p0 : P.p1);
            {
                PhH1_4 h1;
                h1.f.src = (const float *)P.r;
                h1.f.pold = pold;
                h1.f.first = j == 0;
#pragma unroll
                for (int v = 0; v < NR; v++) h1.f.beta[v] = st.beta[v];
                h1.pnew = pnew;
                h1.h = P.hf;
                sweep(h1, acc);
            }
            if (!reduce(acc, sum)) return false;
            if (t0())
                for (int v = 0; v < NR; v++) st.a[v] = st.act[v] ? ArFusedF::div(st.rr[v], sum[v]) : 0.f;
            __syncthreads();
            {
                PhH2_4 h2;
                h2.f.src = pnew;
                h2.f.scale = 1.f;
                h2.z = (float *)P.z;
                h2.r = (float *)P.r;
                h2.first = j == 0;
                h2.h = P.hf;
#pragma unroll
                for (int v = 0; v < NR; v++) h2.a[v] = st.a[v];
                sweep(h2, acc);
            }
            if (!reduce(acc, sum)) return false;
            if (t0()) inner_update(j, sum);
            __syncthreads();
            if (!st.any) break;
        }
        if (t0())
            for (int v = 0; v < NR; v++) st.ih[v] += st.its[v];
        return true;
    }

    // CGNR on S for the right-hand sides still running, from z (P.z) into y
    // (P.y); the others get y = 0.
    __device__ bool s_loop(float gamma)
    {
        float acc[2 * NR], sum[2 * NR];
        {
            PhS0_4 s0;
            s0.f.src = (const float *)P.z;
            s0.f.scale = gamma;
            s0.t = (float *)P.r;
            s0.st = P.tf;
            sweep(s0, acc);
        }
        if (!reduce(acc, sum)) return false;
        if (t0()) {
            float tt0[NR];
            for (int v = 0; v < NR; v++) tt0[v] = sum[v];
            inner_start(tt0, P.tol_s);
        }
        __syncthreads();
        for (int j = 0; j < P.maxit_inner; ++j) {
            float *pnew = (float *)((j & 1) ? P.p1 : P.p0);
            const float *pold = (const float *)((j & 1) ? P.p0 : P.p1);
            {
                PhS1_4 s1;
                s1.f.src = (const float *)P.r;
                s1.f.pold = pold;
                s1.f.first = j == 0;
#pragma unroll
                for (int v = 0; v < NR; v++) s1.f.beta[v] = st.beta[v];
                s1.pnew = pnew;
                s1.u = (float *)P.u;
                s1.sc = P.sf;
                sweep(s1, acc);
            }
            if (!reduce(acc, sum)) return false;
            if (t0())
                for (int v = 0; v < NR; v++) st.a[v] = st.act[v] ? ArFusedF::div(st.rr[v], sum[v]) : 0.f;
            __syncthreads();
            {
                PhS2_4 s2;
                s2.f.src = (const float *)P.u;
                s2.f.scale = 1.f;
                s2.p = pnew;
                s2.y = (float *)P.y;
                s2.t = (float *)P.r;
                s2.first = j == 0;
                s2.st = P.tf;
#pragma unroll
                for (int v = 0; v < NR; v++) s2.a[v] = st.a[v];
                sweep(s2, acc);
            }
            if (!reduce(acc, sum)) return false;
            if (t0()) inner_update(j, sum);
            __syncthreads();
            if (!st.any) break;
        }
        if (t0())
            for (int v = 0; v < NR; v++) st.is[v] += st.its[v];
        return true;
    }

    // Algorithm 1 for each right-hand side, in lockstep; a right-hand side
    // that has stopped keeps its x (its inner solves run with zero steps, so
    // its y is 0).  The final iterate ends in P.xm0 or P.xm1 (*xb_out: 1 =
    // xm1).
    __device__ bool run(int *xb_out)
    {
        const bool leader = vg.b == 0 && threadIdx.x == 0;
        const float gamma = (float)P.co.gamma;
        if (t0())
            for (int v = 0; v < NR; v++) {
                st.r0[v] = st.rel[v] = 0.0;
                st.ih[v] = st.is[v] = 0;
                st.status[v] = ST_NOT_CONVERGED;
                st.kdone[v] = 0;
                st.done[v] = 0;
            }
        __syncthreads();
        Coef7<double> ca;
        ca.d = P.co.a_d;
        ca.e = 0.0;
#pragma unroll
        for (int k = 0; k < 6; k++) ca.c[k] = P.co.a_c[k];
        int xb = 0;
        for (int k = 0;; ++k) {
            double dacc[2 * NR], dsum[2 * NR];
            {
                PhResidual4 ph;
                ph.f.x = xb ? P.xm1 : P.xm0;
                ph.f.y = k > 0 ? (const float *)P.y : nullptr;
                ph.xo = xb ? P.xm0 : P.xm1;
                ph.b = P.bm;
                ph.rs = (float *)P.r;
                ph.cf = ca;
                sweep(ph, dacc);
            }
            if (!reduce(dacc, dsum)) return false;
            xb ^= 1;
            if (t0()) {
                int all = 1;
                for (int v = 0; v < NR; v++) {
                    st.rs2[v] = (float)dsum[NR + v];
                    if (st.done[v]) continue;
                    const double rn = sqrt(dsum[v]);
                    if (k == 0) st.r0[v] = rn;
                    const double rel = st.r0[v] == 0.0 ? 0.0 : rn / st.r0[v];
                    st.rel[v] = rel;
                    double *hist = P.hist + (size_t)v * (P.maxit + 2);
                    if (vg.b == 0) hist[k] = rel;
                    int s = -1;
                    if (rel <= P.tol) s = ST_OK;
                    else if (!(rel == rel) || isinf(rel) || rel > 1e6) s = ST_DIVERGED;
                    else if (P.outer_win > 0 && k >= P.outer_win && rel > 0.99 * __ldcg(hist + (k - P.outer_win)))
                        s = ST_STAGNATED;
                    else if (k >= P.maxit) s = ST_NOT_CONVERGED;
                    if (s >= 0) {
                        st.done[v] = 1;
                        st.status[v] = s;
                        st.kdone[v] = k;
                    } else {
                        all = 0;
                    }
                }
                st.all = all;
            }
            __syncthreads();
            if (st.all) break;
            if (!h_loop()) return false;
            if (!s_loop(gamma)) return false;
        }
        if (leader) {
            for (int v = 0; v < NR; v++) {
                Ctl &c = P.ctl[v];
                c.status = st.status[v];
                c.outer_its = st.kdone[v];
                c.inner_h = st.ih[v];
                c.inner_s = st.is[v];
                c.relres = st.rel[v];
                c.r0 = st.r0[v];
            }
        }
        *xb_out = xb;
        return true;
    }
};

} // namespace gadi

namespace gadi {

// The batched launch with units of four interleaved right-hand sides (one
// system each): the same groups and queues as gadi_batched_kernel.  A
// group's work area holds x (two buffers) and b as [n][4] FP64 and the six
// inner vectors as [n][4] FP32; the unit's right-hand sides and initial
// guesses are gathered into it from the caller's [4][n] arrays, and the final
// iterates scattered back.  Per unit: 4 control blocks (B.ctl + 4 u), 4 x
// B.hist_len history entries of the group, 16 partial sums per block.
__global__ void __launch_bounds__(kThreads, GADI_MIN_BLOCKS) gadi_batched4_kernel(const __grid_constant__ BatchParams B)
{
    const int g = B.block_group[blockIdx.x];
    const int gsize = B.group_size[g];
    const VGrid vg{(int)blockIdx.x - B.group_first[g], gsize};
    GridSync gs;
    gs.counter = B.bar + (size_t)g * 8;
    gs.abort_flag = B.abort_flag;
    gs.nblocks = (unsigned)gsize;
    volatile int *slot = B.group_unit + (size_t)g * 32;
    const bool leader = vg.b == 0 && threadIdx.x == 0;
    const int own_class = B.group_class[g];
    for (;;) {
        if (leader) {
            int u = B.nunits;
            for (int c = own_class; c < B.nclasses && u == B.nunits; c++) {
                const int n_c = B.class_begin[c + 1] - B.class_begin[c];
                if (ld_volatile_int(B.queue + (size_t)c * 32) >= n_c) continue;
                const int i = atomicAdd(B.queue + (size_t)c * 32, 1);
                if (i < n_c) u = B.order[B.class_begin[c] + i];
            }
            if (u < B.nunits) {
                Params &P = B.units[u];
                char *w = B.work + (size_t)g * B.group_work_bytes;
                P.xm0 = (double *)w;
                P.xm1 = (double *)(w + B.slab_d_bytes);
                P.bm = (double *)(w + 2 * B.slab_d_bytes);
                w += 3 * B.slab_d_bytes;
                void **slots[6] = {&P.r, &P.z, &P.p0, &P.p1, &P.y, &P.u};
                for (int i = 0; i < 6; i++) {
                    *slots[i] = w;
                    w += B.slab_bytes;
                }
                P.q = nullptr;
                P.part = B.part + (size_t)16 * B.group_first[g];
                P.bar = B.bar + (size_t)g * 8;
                P.hist = B.hist + (size_t)g * B.hist_len * NR;
                P.ctl = B.ctl + (size_t)NR * u;
                P.abort_flag = B.abort_flag;
                for (int v = 0; v < NR; v++) B.ctl[(size_t)NR * u + v].pad = gsize;
                B.t0[u] = globaltimer_ns();
            }
            *slot = u;
        }
        if (!gs.sync()) return;
        const int u = *slot;
        if (u >= B.nunits) return;
        const Params &P = B.units[u];
        const long long n = P.npts;
        // gather: [4][n] -> [n][4]
        for (long long i = vg.tid(); i < NR * n; i += vg.nthreads()) {
            const long long pt = i >> 2, v = i & 3;
            P.bm[i] = __ldcg(P.b + v * n + pt);
            P.xm0[i] = __ldcg(P.x + v * n + pt);
        }
        if (!gs.sync()) return;
        int xb = 0;
        {
            __shared__ State4 st4;
            Runner4 R(P, vg, st4);
            if (!R.run(&xb)) return;
        }
        if (!gs.sync()) return;
        // scatter the final iterates: [n][4] -> [4][n]
        const double *xf = xb ? P.xm1 : P.xm0;
        for (long long i = vg.tid(); i < NR * n; i += vg.nthreads()) {
            const long long pt = i >> 2, v = i & 3;
            P.x[v * n + pt] = __ldcg(xf + i);
        }
        if (!gs.sync()) return;
        if (leader) B.t1[u] = globaltimer_ns();
    }
}

} // namespace gadi
