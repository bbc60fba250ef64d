"""The slab partition's local products through the CUDA library: each rank
of a 2- or 3-rank plan, run one after another on one GPU with its ghost
planes taken from the full vector (what the halo exchange delivers), must
give the full grid's operator products bit for bit (gadi_apply on extended
sub-grids against gadi_apply on the whole grid, FP64)."""
import numpy as np
import pytest

import paper_2512_21164_gb300 as G
from paper_2512_21164_gb300 import slab
from workloads import conv_diff_2d, conv_diff_3d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2512_21164_gb300 import build
    build.build()


@pytest.mark.parametrize("case", ["2d", "3d"])
@pytest.mark.parametrize("world", [2, 3])
def test_library_slabs_reproduce_the_full_grid(case, world):
    import torch
    p, xt = conv_diff_2d(96, 41, ny=50) if case == "2d" else conv_diff_3d(20, 42)
    x = torch.from_numpy(np.asarray(xt, np.float64) - 0.3).cuda()
    ls = slab.LibraryStencil(p.kind, p.nx, p.ny, p.nz, p.hh, p.beta, p.kappa, p.sigma)
    alpha = 0.37
    try:
        with G.Gadi.from_problem(p) as H:
            full = {}
            for which in (G.OP_A, G.OP_M, G.OP_N):
                y = torch.empty_like(x)
                H.apply(which, x, y)
                full[which] = y
            u_full = alpha * x + full[G.OP_N]
            nu = torch.empty_like(x)
            H.apply(G.OP_N, u_full, nu)
            w_full = alpha * u_full - nu
        for r in range(world):
            plan = slab.plan_for_grid(p.kind, p.nx, p.ny, p.nz, world, r)
            sl = slice(plan.lo * plan.plane_elems, plan.hi * plan.plane_elems)
            for which in (G.OP_A, G.OP_M, G.OP_N):
                y = slab.apply_partitioned(plan, ls.op(which), None, x_ext=slab.extend_from_full(plan, x, 1))
                assert torch.equal(y, full[which][sl]), (r, which)

            def s_ext(v, planes, sign):
                n = ls.op(G.OP_N)(v, planes)
                return alpha * v + sign * n

            w, u = slab.apply_normal_partitioned(plan, lambda v, n: s_ext(v, n, 1.0),
                                                 lambda v, n: s_ext(v, n, -1.0), None,
                                                 p_ext=slab.extend_from_full(plan, x, 2))
            assert torch.equal(u, u_full[sl]) and torch.equal(w, w_full[sl]), r
    finally:
        ls.close()
