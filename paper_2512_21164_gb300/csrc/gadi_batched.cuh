// Batched persistent solve: many independent 2D systems and right-hand sides
// in one cooperative launch.  The grid is split into groups of blocks; each
// group takes (system, right-hand side) units from a device-side queue and runs
// Algorithm 1 on it with the same phases as a single solve (on the group's
// blocks, with the group's own barrier, partial sums and work vectors).  Units
// are queued largest first so the groups finish close together.
#pragma once
#include "gadi_params.h"
#include "gadi_solver.cuh"

namespace gadi {

template <int KIND, int PREC, int WI, int WR, bool DD = false>
__global__ void __launch_bounds__(kThreads, GADI_MIN_BLOCKS) gadi_batched_kernel(const __grid_constant__ BatchParams B)
{
    using SI = StencilImpl<KIND, PREC, WI, WR, DD>;
    const int g = blockIdx.x / B.gsize;
    const VGrid vg{(int)blockIdx.x - g * B.gsize, B.gsize};
    GridSync gs;
    gs.counter = B.bar + (size_t)g * 8;
    gs.abort_flag = B.abort_flag;
    gs.nblocks = (unsigned)B.gsize;
    volatile int *slot = B.group_unit + (size_t)g * 32;
    const bool leader = vg.b == 0 && threadIdx.x == 0;
    for (;;) {
        if (leader) {
            const int u = atomicAdd(B.queue, 1);
            if (u < B.nunits) {
                Params &P = B.units[u];
                char *w = B.work + (size_t)g * B.group_work_bytes;
                P.x1 = (double *)w;
                w += B.slab_d_bytes;
                void **slots[6] = {&P.r, &P.z, &P.p0, &P.p1, &P.y, &P.u};
                for (int i = 0; i < 6; i++) {
                    *slots[i] = w;
                    w += B.slab_bytes;
                }
                P.q = nullptr;
                P.part = B.part + (size_t)g * 4 * B.gsize;
                P.bar = B.bar + (size_t)g * 8;
                P.hist = B.hist + (size_t)g * B.hist_len;
                P.ctl = B.ctl + u;
                P.abort_flag = B.abort_flag;
                B.t0[u] = globaltimer_ns();
            }
            *slot = u;
        }
        if (!gs.sync()) return;
        const int u = *slot;
        if (u >= B.nunits) return;
        const Params &P = B.units[u];
        {
            // (units never take the SM-resident H-solve: a group's blocks share SMs)
            StencilAdapter<SI> I(P, vg);
            Runner<PREC, StencilAdapter<SI>> R(P, I);
            R.run();
        }
        if (!gs.sync()) return;
        // the final iterate into the caller's x
        if (ld_volatile_int(&P.ctl->x_in_x1)) {
            for (long long i = vg.tid(); i < P.nelem; i += vg.nthreads()) P.x[i] = __ldcg(P.x1 + i);
        }
        if (!gs.sync()) return;
        if (leader) B.t1[u] = globaltimer_ns();
    }
}

} // namespace gadi
