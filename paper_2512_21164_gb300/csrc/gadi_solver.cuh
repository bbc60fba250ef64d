// Algorithm 1 control loop (shared by every operator class) and the CSR
// implementation of the phase interface.
#pragma once
#include "gadi_kernel.cuh"

namespace gadi {

// ---------------------------------------------------------------------------
// elementwise helpers shared by all classes
// ---------------------------------------------------------------------------
template <int PREC>
__device__ void phase_norm2(const void *v, long long m, typename AccT<PREC>::T (&acc)[2], VGrid vg)
{
    using PT = Prec<PREC>;
    using S = typename PT::S;
    using AT = typename AccT<PREC>::T;
    const S *s = (const S *)v;
    AT a = AT(0);
    for (long long i = vg.tid(); i < m; i += vg.nthreads()) {
        const AT x = (AT)PT::ld(s[i]);
        a += x * x;
    }
    acc[0] = a;
    acc[1] = AT(0);
}

template <int PREC>
__device__ void phase_zero(void *v, long long m, VGrid vg)
{
    using S = typename Prec<PREC>::S;
    S *s = (S *)v;
    for (long long i = vg.tid(); i < m; i += vg.nthreads()) s[i] = S(0);
}

// ---------------------------------------------------------------------------
// CSR implementation: one thread per row, grid-stride.  Gathers need the
// whole input vector, so phases that gather from a vector written in the same
// phase split at an internal grid barrier.
// ---------------------------------------------------------------------------
template <int PREC, bool DD = false>
struct CsrImpl {
    using PT = Prec<PREC>;
    using S = typename PT::S;
    using C = typename PT::C;
    using A = typename InnerAr<PREC>::T;
    using AT = typename AccT<PREC>::T;
    static constexpr int K = 1;
    static constexpr bool RESIDENT = false;
    const Params &P;
    VGrid vg;
    int n;
    __device__ CsrImpl(const Params &p, VGrid g) : P(p), vg(g) { n = (int)p.npts; }

    __device__ long long i0() const { return vg.tid(); }
    __device__ long long di() const { return vg.nthreads(); }

    template <class VT, class XT, class AR>
    __device__ VT spmv_row(const int *rp, const int *cl, const VT *val, const XT *x, int i) const
    {
        VT s = VT(0);
        for (int k = rp[i]; k < rp[i + 1]; k++) s = AR::madd(val[k], (VT)ldx(x, cl[k]), s);
        return s;
    }
    template <class T> __device__ static auto ldx(const T *x, int j)
    {
        if constexpr (sizeof(T) == 8) return __ldcg(x + j);
        else return PT::ld(x[j]);
    }
    template <class VT, class VP> __device__ static VT ldv(const VP *v, int k)
    {
        if constexpr (sizeof(VP) == 8) return (VT)v[k];
        else return (VT)PT::ld(v[k]);
    }
    // Sparse products over the rows, RB rows per thread at a time (rows i,
    // i + di, ..., a grid stride apart): their row pointers, indices and
    // gathers are independent loads, so a thread keeps RB rows' loads in
    // flight instead of one chain of dependent loads.  Each row still sums
    // its entries in CSR order.  body(row, sum) consumes each row's result.
    // (2048^2 as CSR: 4 rows 10.08 s, 6 rows 9.82 s, 8 rows 9.99 s)
    static constexpr int RB = 6;
    template <class VT, class XT, class AR, class VP, class Body>
    __device__ void spmv_loop(const int *rp, const int *cl, const VP *val, const XT *x, Body body) const
    {
        const long long step = di();
        for (long long i = i0(); i < n; i += RB * step) {
            int b[RB], e[RB], len = 0;
            VT sum[RB];
#pragma unroll
            for (int r = 0; r < RB; r++) {
                const long long row = i + r * step;
                b[r] = row < n ? rp[row] : 0;
                e[r] = row < n ? rp[row + 1] : 0;
                sum[r] = VT(0);
                len = max(len, e[r] - b[r]);
            }
            for (int k = 0; k < len; k++) {
#pragma unroll
                for (int r = 0; r < RB; r++)
                    if (b[r] + k < e[r])
                        sum[r] = AR::madd(ldv<VT>(val, b[r] + k), (VT)ldx(x, cl[b[r] + k]), sum[r]);
            }
#pragma unroll
            for (int r = 0; r < RB; r++) {
                const long long row = i + r * step;
                if (row < n) body(row, sum[r]);
            }
        }
    }

    __device__ bool residual(const double *xin, const S *y, double *xout, double (&acc)[2],
                             const GridSync &gs) const
    {
        for (long long i = i0(); i < n; i += di())
            xout[i] = y ? __dadd_rn(xin[i], PT::to_f64(y[i])) : xin[i];
        if (!gs.sync()) return false;
        double a0 = 0.0, a1 = 0.0;
        S *rs = (S *)P.r;
        if constexpr (!DD) {
            spmv_loop<double, double, ArFusedD>(P.rowptr, P.col, P.aval, (const double *)xout,
                                                [&](long long i, double ax) {
                const double r = __dsub_rn(P.b[i], ax);
                const S sv = PT::from_f64(r);
                a0 = fma(r, r, a0);
                rs[i] = sv;
                const double d = PT::to_f64(sv);
                a1 = fma(d, d, a1);
                if (P.r_out) P.r_out[i] = r;
            });
            acc[0] = a0;
            acc[1] = a1;
            return true;
        }
        for (long long i = i0(); i < n; i += di()) {
            double r, rl = 0.0;
            S sv;
            if constexpr (DD) { // double-FP64: b, then -a_ik x_k in row order (as the stencil phase)
                double hi = P.b[i], lo = 0.0;
                for (int k = P.rowptr[i]; k < P.rowptr[i + 1]; k++)
                    dd_sub_term(hi, lo, P.aval[k], __ldcg(xout + P.col[k]));
                two_sum(hi, lo, r, rl);
                sv = PT::from_f64x2(r, rl);
            } else {
                const double ax = spmv_row<double, double, ArFusedD>(P.rowptr, P.col, P.aval, xout, (int)i);
                r = __dsub_rn(P.b[i], ax);
                sv = PT::from_f64(r);
            }
            a0 = fma(r, r, a0);
            rs[i] = sv;
            const double d = PT::to_f64(sv);
            a1 = fma(d, d, a1);
            if (P.r_out) P.r_out[i] = r;
            if constexpr (DD)
                if (P.r_lo_out) P.r_lo_out[i] = rl;
        }
        acc[0] = a0;
        acc[1] = a1;
        return true;
    }
    __device__ bool apply(const double *x, double *yout, const GridSync &) const
    {
        // op selection is done on the host by pointing rowptr/col/aval at
        // the operator to apply
        spmv_loop<double, double, ArFusedD>(P.rowptr, P.col, P.aval, x,
                                            [&](long long i, double v) { yout[i] = v; });
        return true;
    }
    __device__ bool h1(bool first, C beta, const S *pold, S *pnew, AT (&acc)[2], const GridSync &gs) const
    {
        const S *r = (const S *)P.r;
        for (long long i = i0(); i < n; i += di()) {
            C v = PT::ld(r[i]);
            if (!first) v = A::madd(beta, PT::ld(pold[i]), v);
            pnew[i] = PT::st(v);
        }
        if (!gs.sync()) return false;
        AT a = AT(0);
        C *q = (C *)P.q;
        const S *hv = (const S *)P.hval;
        spmv_loop<C, S, A>(P.mrowptr, P.mcol, hv, (const S *)pnew, [&](long long i, C s) {
            q[i] = s;
            a += (AT)PT::ld(pnew[i]) * (AT)s;
        });
        acc[0] = a;
        acc[1] = AT(0);
        return true;
    }
    __device__ bool h2(bool first, C a_, const S *p, AT (&acc)[2], const GridSync &) const
    {
        S *z = (S *)P.z, *r = (S *)P.r;
        const C *q = (const C *)P.q;
        AT a = AT(0);
        for (long long i = i0(); i < n; i += di()) {
            const C pp = PT::ld(p[i]);
            z[i] = PT::st(first ? A::mul(a_, pp) : A::madd(a_, pp, PT::ld(z[i])));
            const S rn = PT::st(A::madd(-a_, q[i], PT::ld(r[i])));
            r[i] = rn;
            const AT rr = (AT)PT::ld(rn);
            a += rr * rr;
        }
        acc[0] = a;
        acc[1] = AT(0);
        return true;
    }
    __device__ bool s0(C gamma, AT (&acc)[2], const GridSync &gs) const
    {
        const S *z = (const S *)P.z;
        S *g = (S *)P.u;
        for (long long i = i0(); i < n; i += di()) g[i] = PT::st(A::mul(gamma, PT::ld(z[i])));
        if (!gs.sync()) return false;
        S *t = (S *)P.r;
        const S *tv = (const S *)P.tval;
        AT a = AT(0);
        spmv_loop<C, S, A>(P.mrowptr, P.mcol, tv, (const S *)g, [&](long long i, C s) {
            const S ts = PT::st(s);
            t[i] = ts;
            const AT x = (AT)PT::ld(ts);
            a += x * x;
        });
        acc[0] = a;
        acc[1] = AT(0);
        return true;
    }
    __device__ bool s1(bool first, C beta, const S *pold, S *pnew, AT (&acc)[2], const GridSync &gs) const
    {
        const S *t = (const S *)P.r;
        for (long long i = i0(); i < n; i += di()) {
            C v = PT::ld(t[i]);
            if (!first) v = A::madd(beta, PT::ld(pold[i]), v);
            pnew[i] = PT::st(v);
        }
        if (!gs.sync()) return false;
        S *u = (S *)P.u;
        const S *sv = (const S *)P.sval;
        AT a = AT(0);
        spmv_loop<C, S, A>(P.mrowptr, P.mcol, sv, (const S *)pnew, [&](long long i, C s) {
            const S us = PT::st(s);
            u[i] = us;
            const AT x = (AT)PT::ld(us);
            a += x * x;
        });
        acc[0] = a;
        acc[1] = AT(0);
        return true;
    }
    __device__ bool s2(bool first, C a_, const S *p, AT (&acc)[2], const GridSync &) const
    {
        const S *u = (const S *)P.u;
        const S *tv = (const S *)P.tval;
        S *y = (S *)P.y, *t = (S *)P.r;
        AT a = AT(0);
        spmv_loop<C, S, A>(P.mrowptr, P.mcol, tv, u, [&](long long i, C w) {
            const C pp = PT::ld(p[i]);
            y[i] = PT::st(first ? A::mul(a_, pp) : A::madd(a_, pp, PT::ld(y[i])));
            const S tn = PT::st(A::madd(-a_, w, PT::ld(t[i])));
            t[i] = tn;
            const AT x = (AT)PT::ld(tn);
            a += x * x;
        });
        acc[0] = a;
        acc[1] = AT(0);
        return true;
    }
    __device__ void s_pointwise(C) const {}
    // (the SM-resident H-solve exists for the 2D stencil class only)
    struct ResRing {};
    static constexpr bool TMEM = false;
    __device__ void hflush(bool) const {}
    __device__ void s0r(C, bool, AT (&acc)[2]) const { acc[0] = acc[1] = AT(0); }
    __device__ void s1r(int, C, AT (&acc)[2]) const { acc[0] = acc[1] = AT(0); }
    __device__ void s2r(bool, C, AT (&acc)[2]) const { acc[0] = acc[1] = AT(0); }
    __device__ void sflush() const {}
    __device__ void h1r(int, C, AT (&acc)[2]) const { acc[0] = acc[1] = AT(0); }
    __device__ void h2pre(bool, ResRing &) const {}
    __device__ void h2r(bool, C, AT (&acc)[2], ResRing &) const { acc[0] = acc[1] = AT(0); }
};

// Adapter giving the stencil implementation the same (bool-returning,
// barrier-taking) interface as the CSR one.  RES: 0 streaming H-solve,
// 1 SM-resident p (z and r in global memory / L2), 2 SM-resident p with z
// and r in tensor memory.
template <class SI, int RES = 0>
struct StencilAdapter {
    using S = typename SI::S;
    using C = typename SI::C;
    using A = typename SI::A;
    using AT = typename SI::AT;
    static constexpr int K = SI::K;
    // the SM-resident H-solve is compiled in where it exists and RES allows
    static constexpr bool RESIDENT = SI::RES_OK && RES >= 1;
    static constexpr bool TMEM = SI::TM_OK && RES == 2;
    SI si;
    VGrid vg;
    __device__ StencilAdapter(const Params &p, VGrid g) : si(p, g), vg(g) {}
    __device__ bool residual(const double *xin, const S *y, double *xout, double (&acc)[2],
                             const GridSync &) const
    {
        si.residual(xin, y, xout, acc);
        return true;
    }
    __device__ bool apply(const double *x, double *yout, const GridSync &) const
    {
        si.apply(x, yout);
        return true;
    }
    __device__ bool h1(bool first, C beta, const S *pold, S *pnew, AT (&acc)[2], const GridSync &gs) const
    {
        if constexpr (SI::SPLIT_P) {
            si.p_update(first, beta, pold, pnew);
            if (!gs.sync()) return false;
            si.h1_split(pnew, acc);
        } else {
            si.h1(first, beta, pold, pnew, acc);
        }
        return true;
    }
    __device__ bool h2(bool first, C a, const S *p, AT (&acc)[2], const GridSync &) const
    {
        si.h2(first, a, p, acc);
        return true;
    }
    __device__ bool s0(C gamma, AT (&acc)[2], const GridSync &) const
    {
        si.s0(gamma, acc);
        return true;
    }
    __device__ bool s1(bool first, C beta, const S *pold, S *pnew, AT (&acc)[2], const GridSync &gs) const
    {
        if constexpr (SI::SPLIT_P) {
            si.p_update(first, beta, pold, pnew);
            if (!gs.sync()) return false;
            si.s1_split(pnew, acc);
        } else {
            si.s1(first, beta, pold, pnew, acc);
        }
        return true;
    }
    __device__ bool s2(bool first, C a, const S *p, AT (&acc)[2], const GridSync &) const
    {
        si.s2(first, a, p, acc);
        return true;
    }
    __device__ void s_pointwise(C gamma) const { si.s_pointwise(gamma); }
    using ResRing = typename SI::ResRing;
    __device__ void h1r(int j, C beta, AT (&acc)[2]) const
    {
        if constexpr (TMEM)
            si.h1_tm(j, beta, acc);
        else
            si.h1_res(j, beta, acc);
    }
    __device__ void h2pre(bool first, ResRing &q) const
    {
        if constexpr (!TMEM) si.h2_res_pre(first, q);
    }
    __device__ void h2r(bool first, C a, AT (&acc)[2], ResRing &q) const
    {
        if constexpr (TMEM)
            si.h2_tm(first, a, acc);
        else
            si.h2_res(first, a, acc, q);
    }
    __device__ void hflush(bool edges_only) const { si.h_flush_tm(edges_only); }
    __device__ void s0r(C gamma, bool z_tm, AT (&acc)[2]) const { si.s0_tm(gamma, z_tm, acc); }
    __device__ void s1r(int j, C beta, AT (&acc)[2]) const { si.s1_tm(j, beta, acc); }
    __device__ void s2r(bool first, C a, AT (&acc)[2]) const { si.s2_tm(first, a, acc); }
    __device__ void sflush() const { si.s_flush_tm(); }
};

// ---------------------------------------------------------------------------
// the control loop
// ---------------------------------------------------------------------------
// largest value of type C not above x (so that c <= x in double is c <= floor_to(x) in C)
template <class C> __device__ __forceinline__ C floor_to(double x);
template <> __device__ __forceinline__ float floor_to<float>(double x) { return __double2float_rd(x); }
template <> __device__ __forceinline__ double floor_to<double>(double x) { return x; }

template <int PREC, class Impl>
struct Runner {
    using PT = Prec<PREC>;
    using S = typename PT::S;
    using C = typename PT::C;
    using A = typename InnerAr<PREC>::T;
    using AT = typename AccT<PREC>::T;
    const Params &P;
    const Impl &I;
    GridSync gs;
    int slot = 0;

    __device__ Runner(const Params &p, const Impl &i) : P(p), I(i)
    {
        gs.counter = p.bar;
        gs.abort_flag = p.abort_flag;
        gs.nblocks = (unsigned)i.vg.n;
    }

    // grid-wide sums of two per-thread partials; every block gets the same
    // totals.  Two slots alternate so a fast block cannot overwrite partials a
    // slow block is still reading.
    template <class RT>
    __device__ bool reduce(const RT (&acc)[2], RT (&out)[2])
    {
        const int G = I.vg.n;
        RT *part = reinterpret_cast<RT *>(P.part + (size_t)slot * 2 * G);
        block_partials_write<2, RT>(acc, part, G, I.vg.b);
        if (!gs.sync()) return false;
        grid_partials_sum<2, RT>(part, G, out);
        slot ^= 1;
        return true;
    }
    // reduce() in two halves: between them the block may do work that reads
    // nothing other blocks wrote since the previous barrier
    template <class RT>
    __device__ unsigned long long reduce_begin(const RT (&acc)[2])
    {
        const int G = I.vg.n;
        RT *part = reinterpret_cast<RT *>(P.part + (size_t)slot * 2 * G);
        block_partials_write<2, RT>(acc, part, G, I.vg.b);
        return gs.arrive();
    }
    template <class RT>
    __device__ bool reduce_end(unsigned long long arrived, RT (&out)[2])
    {
        if (!gs.wait(arrived)) return false;
        grid_partials_sum<2, RT>(reinterpret_cast<const RT *>(P.part + (size_t)slot * 2 * I.vg.n), I.vg.n, out);
        slot ^= 1;
        return true;
    }

    // CG on H = alpha I + M (right-hand side already in P.r, ||rhs||^2 = rr0).
    // Returns iterations, or -1 if a barrier gave up.
    __device__ int h_loop(C rr)
    {
        const long long m = P.nelem;
        if (rr == C(0)) {
            phase_zero<PREC>(P.z, m, I.vg);
            return gs.sync() ? 0 : -1;
        }
        // stop when rn <= tol^2 rr0 (compared in double, evaluated in C)
        const C thr = floor_to<C>(P.tol_h * P.tol_h * (double)rr);
        C beta = C(0), best = rr;
        int since = 0, its = 0;
        AT acc[2], sum[2];
        for (int j = 0; j < P.maxit_inner; ++j) {
            S *pnew = (S *)((j & 1) ? P.p1 : P.p0);
            const S *pold = (const S *)((j & 1) ? P.p0 : P.p1);
            // the resident instantiation runs only with P.resident set
            if constexpr (Impl::RESIDENT) {
                I.h1r(j, beta, acc);
                // the first rows of z and r the update needs are loaded
                // while the barrier of p.(Hp) is open
                const unsigned long long arrived = reduce_begin(acc);
                typename Impl::ResRing ring;
                I.h2pre(j == 0, ring);
                if (!reduce_end(arrived, sum)) return -1;
                I.h2r(j == 0, A::div(rr, (C)sum[0]), acc, ring);
            } else {
                if (!I.h1(j == 0, beta, pold, pnew, acc, gs)) return -1;
                if (!reduce(acc, sum)) return -1;
                if (!I.h2(j == 0, A::div(rr, (C)sum[0]), pnew, acc, gs)) return -1;
            }
            if (!reduce(acc, sum)) return -1;
            const C rn = (C)sum[0];
            its = j + 1;
            if (rn <= thr) break;
            if (!(rn == rn)) break;
            if (rn < best) {
                best = rn;
                since = 0;
            } else if (P.inner_stag > 0 && ++since >= P.inner_stag) {
                break;
            }
            beta = A::div(rn, rr);
            rr = rn;
        }
        if constexpr (Impl::TMEM) {
            // z leaves tensor memory; the S-solve reads it across blocks
            // (the resident S-solve only the rows the neighbours' halo
            // needs: it takes its own rows from tensor memory)
            if (its > 0) {
                I.hflush(P.s_resident && P.mode == MODE_SOLVE);
                if (!gs.sync()) return -1;
            }
        }
        return its;
    }

    // CGNR on S with p in shared memory and t, y in tensor memory (the
    // TMEM kernel, P.s_resident); z_tm: z of the own rows is in tensor
    // memory (the H-solve ran), else in global memory
    __device__ int s_loop_res(C gamma, bool z_tm)
    {
        const long long m = P.nelem;
        AT acc[2], sum[2];
        I.s0r(gamma, z_tm, acc);
        if (!reduce(acc, sum)) return -1;
        C tt = (C)sum[0];
        if (tt == C(0)) {
            phase_zero<PREC>(P.y, m, I.vg);
            return gs.sync() ? 0 : -1;
        }
        const C thr = floor_to<C>(P.tol_s * P.tol_s * (double)tt);
        C beta = C(0), best = tt;
        int since = 0, its = 0;
        for (int j = 0; j < P.maxit_inner; ++j) {
            I.s1r(j, beta, acc);
            if (!reduce(acc, sum)) return -1;
            const C a = A::div(tt, (C)sum[0]);
            I.s2r(j == 0, a, acc);
            if (!reduce(acc, sum)) return -1;
            const C tn = (C)sum[0];
            its = j + 1;
            if (tn <= thr) break;
            if (!(tn == tn)) break;
            if (tn < best) {
                best = tn;
                since = 0;
            } else if (P.inner_stag > 0 && ++since >= P.inner_stag) {
                break;
            }
            beta = A::div(tn, tt);
            tt = tn;
        }
        // y leaves tensor memory; the next residual reads it across blocks
        if (its > 0) {
            I.sflush();
            if (!gs.sync()) return -1;
        }
        return its;
    }

    // S-solve from z (P.z) into y (P.y).  Returns iterations or -1.
    // z_tm: the H-solve left z of the own rows in tensor memory.
    __device__ int s_loop(C gamma, bool z_tm = false)
    {
        if constexpr (Impl::TMEM) {
            if (P.s_resident) return s_loop_res(gamma, z_tm);
        }
        const long long m = P.nelem;
        if (Impl::K == 2 && P.pointwise) {
            I.s_pointwise(gamma);
            return gs.sync() ? 1 : -1;
        }
        AT acc[2], sum[2];
        if (!I.s0(gamma, acc, gs) || !reduce(acc, sum)) return -1;
        C tt = (C)sum[0];
        if (tt == C(0)) {
            phase_zero<PREC>(P.y, m, I.vg);
            return gs.sync() ? 0 : -1;
        }
        const C thr = floor_to<C>(P.tol_s * P.tol_s * (double)tt);
        C beta = C(0), best = tt;
        int since = 0, its = 0;
        for (int j = 0; j < P.maxit_inner; ++j) {
            S *pnew = (S *)((j & 1) ? P.p1 : P.p0);
            const S *pold = (const S *)((j & 1) ? P.p0 : P.p1);
            if (!I.s1(j == 0, beta, pold, pnew, acc, gs) || !reduce(acc, sum)) return -1;
            const C a = A::div(tt, (C)sum[0]);
            if (!I.s2(j == 0, a, pnew, acc, gs) || !reduce(acc, sum)) return -1;
            const C tn = (C)sum[0];
            its = j + 1;
            if (tn <= thr) break;
            if (!(tn == tn)) break;
            if (tn < best) {
                best = tn;
                since = 0;
            } else if (P.inner_stag > 0 && ++since >= P.inner_stag) {
                break;
            }
            beta = A::div(tn, tt);
            tt = tn;
        }
        return its;
    }

    __device__ void run()
    {
        const bool leader = I.vg.b == 0 && threadIdx.x == 0;
        double dacc[2], dsum[2];
        if (P.mode == MODE_APPLY) {
            I.apply(P.ax_in, P.ax_out, gs);
            return;
        }
        if (P.mode == MODE_RESIDUAL) {
            if (!I.residual(P.x, (const S *)P.y, P.x1, dacc, gs) || !reduce(dacc, dsum)) return;
            if (leader) {
                P.ctl->rnorm = sqrt(dsum[0]);
                P.ctl->status = ST_OK;
            }
            return;
        }
        if (P.mode == MODE_SOLVE_H) {
            AT acc[2], sum[2];
            phase_norm2<PREC>(P.r, P.nelem, acc, I.vg);
            if (!reduce(acc, sum)) return;
            const int its = h_loop((C)sum[0]);
            if (leader && its >= 0) {
                P.ctl->inner_h = its;
                P.ctl->status = ST_OK;
            }
            return;
        }
        if (P.mode == MODE_SOLVE_S) {
            const int its = s_loop((C)P.co.gamma);
            if (leader && its >= 0) {
                P.ctl->inner_s = its;
                P.ctl->status = ST_OK;
            }
            return;
        }
        // MODE_SOLVE: Algorithm 1
        double r0 = 0.0, rel = 0.0;
        long long ih = 0, is = 0;
        int status = ST_NOT_CONVERGED, k = 0, xb = 0;
        const C gamma = (C)P.co.gamma;
        for (k = 0;; ++k) {
            const double *xin = xb ? P.x1 : P.x;
            double *xout = xb ? P.x : P.x1;
            if (!I.residual(xin, k > 0 ? (const S *)P.y : nullptr, xout, dacc, gs) || !reduce(dacc, dsum)) return;
            xb ^= 1;
            const double rn = sqrt(dsum[0]);
            if (k == 0) r0 = rn;
            rel = r0 == 0.0 ? 0.0 : rn / r0; // non-finite r0: NaN, hence DIVERGED
            if (leader) P.hist[k] = rel;
            if (rel <= P.tol) {
                status = ST_OK;
                break;
            }
            if (!(rel == rel) || isinf(rel) || rel > 1e6) {
                status = ST_DIVERGED;
                break;
            }
            if (P.outer_win > 0 && k >= P.outer_win && rel > 0.99 * __ldcg(P.hist + (k - P.outer_win))) {
                status = ST_STAGNATED;
                break;
            }
            if (k >= P.maxit) {
                status = ST_NOT_CONVERGED;
                break;
            }
            const int a = h_loop((C)dsum[1]);
            if (a < 0) return;
            ih += a;
            const int b = s_loop(gamma, a > 0);
            if (b < 0) return;
            is += b;
        }
        if (leader) {
            P.ctl->status = status;
            P.ctl->outer_its = k;
            P.ctl->inner_h = ih;
            P.ctl->inner_s = is;
            P.ctl->relres = rel;
            P.ctl->r0 = r0;
            P.ctl->x_in_x1 = xb;
        }
    }
};

// RES = 1: the instantiation with the SM-resident H-solve (2D real class,
// FP32/BF16, 16-byte path), a kernel of its own so that its register needs
// leave the streaming kernels' code alone; RES = 2: the same with z and r
// of the H-solve in tensor memory.  The RES = 2 kernel allocates all 512
// TMEM columns of its SM for the launch (it runs one block per SM: its
// register file use leaves room for no other block) and frees them on
// every way out.
template <int KIND, int PREC, int WI, int WR, int RES = 0, bool DD = false>
__global__ void __launch_bounds__(kThreads, GADI_MIN_BLOCKS) gadi_stencil_kernel(const __grid_constant__ Params P)
{
    using Ad = StencilAdapter<StencilImpl<KIND, PREC, WI, WR, DD, RES == 2 ? 1 : (KIND == K_2D5 && RES == 0 ? 2 : 0)>,
                              RES>;
    Ad I(P, whole_grid());
    if constexpr (Ad::TMEM) {
        __shared__ unsigned s_tm;
        const bool w0 = threadIdx.x < 32;
        if (w0) {
            tmem_alloc(&s_tm, 512u);
            tmem_relinquish();
        }
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        I.si.tm = s_tm;
        if (I.si.tm_fits()) {
            Runner<PREC, Ad> R(P, I);
            R.run();
        } else if (threadIdx.x == 0) {
            atomicExch(P.abort_flag, 1); // the host refuses such shapes first
        }
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        if (w0) tmem_dealloc(s_tm, 512u);
    } else {
        Runner<PREC, Ad> R(P, I);
        R.run();
    }
}

template <int PREC, bool DD = false>
__global__ void __launch_bounds__(kThreads, GADI_MIN_BLOCKS) gadi_csr_kernel(const __grid_constant__ Params P)
{
    CsrImpl<PREC, DD> I(P, whole_grid());
    Runner<PREC, CsrImpl<PREC, DD>> R(P, I);
    R.run();
}

} // namespace gadi
