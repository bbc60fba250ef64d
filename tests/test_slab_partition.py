"""Slab partitioning of one system over two and three ranks (gloo on CPU): the plan,
the halo exchange and the partitioned operator products reproduce the
undivided grid's products bit for bit, and a partitioned CG on H (one halo
exchange per product, two all-reduces per iteration) matches the oracle's CG.

The local stencil of each rank is the oracle's FP64 operator on the rank's
extended sub-grid (the tests may use the oracle; on GPUs the library's
gadi_apply plays that part).  The partition, the exchange and the reductions
are the product's (paper_2512_21164_gb300.slab)."""
import os
import socket

import numpy as np
import pytest

from paper_2512_21164_gb300 import slab


def test_plan_is_balanced_and_covers_the_grid():
    for planes, world in [(10, 2), (11, 3), (7, 7), (512, 8)]:
        plans = [slab.make_plan(planes, 5, world, r) for r in range(world)]
        assert plans[0].lo == 0 and plans[-1].hi == planes
        for a, b in zip(plans, plans[1:]):
            assert a.hi == b.lo
        sizes = [p.own for p in plans]
        assert max(sizes) - min(sizes) <= 1
        assert plans[0].prev is None and plans[-1].next is None
    with pytest.raises(ValueError):
        slab.make_plan(3, 5, 4, 0)
    p3 = slab.plan_for_grid(1, 6, 5, 9, 2, 1)
    assert p3.plane_elems == 30 and (p3.lo, p3.hi) == (4, 9)
    pc = slab.plan_for_grid(2, 6, 8, 1, 2, 0)
    assert pc.plane_elems == 12 and (pc.lo, pc.hi) == (0, 4)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _sub_problem(p, planes):
    """The same stencil on a sub-grid of `planes` planes along the split axis
    (same h: the full grid's)."""
    from workloads import K_3D7, Problem
    if p.kind == K_3D7:
        return Problem(p.kind, p.nx, p.ny, planes, p.hh, p.beta, p.kappa, p.sigma)
    return Problem(p.kind, p.nx, planes, 1, p.hh, p.beta, p.kappa, p.sigma)


def _cases():
    from workloads import complex_rd, conv_diff_2d, conv_diff_3d
    return [conv_diff_2d(23, 31, ny=17), conv_diff_3d(7, 32), complex_rd(9, 33)]


def _rank_main(rank, world, port, results):
    import torch
    import torch.distributed as dist

    import oracle as O
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = {}
    try:
        for ci, (p, xt) in enumerate(_cases()):
            orc = O.Oracle(p)
            plan = slab.plan_for_grid(p.kind, p.nx, p.ny, p.nz, world, rank)
            pe = plan.plane_elems
            x = np.asarray(xt, np.float64) - 0.3
            x_own = torch.from_numpy(x[plan.lo * pe: plan.hi * pe].copy())
            for which in (O.OP_A, O.OP_M, O.OP_N):
                def local(v_ext, planes, which=which):
                    return torch.from_numpy(O.Oracle(_sub_problem(p, planes)).apply(which, v_ext.numpy()))
                y = slab.apply_partitioned(plan, local, x_own).numpy()
                full = orc.apply(which, x)[plan.lo * pe: plan.hi * pe]
                out[(ci, which)] = bool(np.array_equal(y, full))
            # S^T (S p) with two ghost planes, S = alpha I + N
            alpha = 0.37

            def s_ext(v, planes, sign):
                sub = O.Oracle(_sub_problem(p, planes))
                return torch.from_numpy(alpha * v.numpy() + sign * sub.apply(O.OP_N, v.numpy()))

            w, u = slab.apply_normal_partitioned(plan, lambda v, n: s_ext(v, n, 1.0),
                                                 lambda v, n: s_ext(v, n, -1.0), x_own)
            u_full = alpha * x + orc.apply(O.OP_N, x)
            w_full = alpha * u_full - orc.apply(O.OP_N, u_full)
            sl = slice(plan.lo * pe, plan.hi * pe)
            out[(ci, "StS")] = bool(np.array_equal(w.numpy(), w_full[sl]) and np.array_equal(u.numpy(), u_full[sl]))
            # a partitioned CG on H = alpha I + M (FP64): one exchange per
            # product, the two sums of each iteration by all-reduce
            if ci == 0:
                rs = torch.from_numpy(x[sl].copy())
                a_h = 0.2

                def h_ext(v, planes):
                    return torch.from_numpy(a_h * v.numpy() + O.Oracle(_sub_problem(p, planes)).apply(O.OP_M, v.numpy()))

                z = torch.zeros_like(rs)
                r = rs.clone()
                (rr,) = slab.allreduce_sum([float(torch.dot(r, r))])
                rr0, its = rr, 0
                pdir = r.clone()
                for j in range(200):
                    if j:
                        pdir = r + beta * pdir
                    q = slab.apply_partitioned(plan, h_ext, pdir)
                    (pq,) = slab.allreduce_sum([float(torch.dot(pdir, q))])
                    a = rr / pq
                    z = z + a * pdir
                    r = r - a * q
                    (rn,) = slab.allreduce_sum([float(torch.dot(r, r))])
                    its = j + 1
                    if rn <= 1e-20 * rr0:
                        break
                    beta, rr = rn / rr, rn
                zo, it_o = orc.solve_h(a_h, O.FP64, x, 1e-10, 200, 0)
                out["cg_its"] = (its, it_o)
                out["cg_err"] = float(np.max(np.abs(z.numpy() - zo[sl])) / np.max(np.abs(zo)))
    finally:
        dist.destroy_process_group()
    results[rank] = out


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_reproduce_the_undivided_grid(world):
    """world = 3: the middle rank exchanges ghost planes with both neighbours."""
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    results = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, results), nprocs=world, join=True)
    assert set(results.keys()) == set(range(world))
    for rank in range(world):
        res = dict(results[rank])
        for key, ok in res.items():
            if isinstance(key, tuple):
                assert ok, (rank, key)
        its, it_o = res["cg_its"]
        assert abs(its - it_o) <= 1, (its, it_o)
        assert res["cg_err"] <= 1e-12, res["cg_err"]
