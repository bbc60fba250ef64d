// Batched persistent solve: many independent 2D systems and right-hand sides
// in one cooperative launch.  The grid is split into groups of blocks; each
// group takes (system, right-hand side) units from a device-side queue and runs
// Algorithm 1 on it with the same phases as a single solve (on the group's
// blocks, with the group's own barrier, partial sums and work vectors).  Units
// are queued largest first so the groups finish close together.  RES = 1: the
// units' CG on H keeps its direction p in shared memory (the SM-resident
// H-solve of the single solve, on the group's blocks: block b of a group of G
// owns rows [b ny / G, (b+1) ny / G) of the unit), the launch's dynamic shared
// memory sized by the host for the largest share a group may take.
#pragma once
#include "gadi_params.h"
#include "gadi_solver.cuh"

namespace gadi {

template <int KIND, int PREC, int WI, int WR, bool DD = false, int RES = 0>
__global__ void __launch_bounds__(kThreads, GADI_MIN_BLOCKS) gadi_batched_kernel(const __grid_constant__ BatchParams B)
{
    using SI = StencilImpl<KIND, PREC, WI, WR, DD>;
    using Ad = StencilAdapter<SI, RES>;
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
            // the group's own class first, then the classes of smaller
            // systems (classes are sorted by system size, largest first): a
            // group never takes a unit larger than those it was sized for,
            // nor one of a class whose size limits exclude the group's size
            int u = B.nunits;
            for (int k = own_class; k < B.nclasses && u == B.nunits; k++) {
                const int c = k;
                if (gsize < B.class_gmin[c] || gsize > B.class_gmax[c]) continue;
                const int n_c = B.class_begin[c + 1] - B.class_begin[c];
                if (ld_volatile_int(B.queue + (size_t)c * 32) >= n_c) continue;
                const int i = atomicAdd(B.queue + (size_t)c * 32, 1);
                if (i < n_c) u = B.order[B.class_begin[c] + i];
            }
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
                P.part = B.part + (size_t)4 * B.group_first[g];
                P.bar = B.bar + (size_t)g * 8;
                P.hist = B.hist + (size_t)g * B.hist_len;
                P.ctl = B.ctl + u;
                P.abort_flag = B.abort_flag;
                B.ctl[u].pad = gsize; // reported as the unit's block count
                B.t0[u] = globaltimer_ns();
            }
            *slot = u;
        }
        if (!gs.sync()) return;
        const int u = *slot;
        if (u >= B.nunits) return;
        const Params &P = B.units[u];
        {
            Ad I(P, vg);
            Runner<PREC, Ad> R(P, I);
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
