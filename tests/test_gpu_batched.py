"""The batched persistent solve (many systems and right-hand sides in one
launch) against the CPU oracle: every (system, right-hand side) unit must
reach the oracle's outcome for that system, within the outer-iteration band
of the single-system tests, and match the single-system GPU solve."""
import numpy as np
import pytest

import oracle as O
import paper_2512_21164_gb300 as G
from helpers import BF16, FP32, FP64, dev64
from workloads import SplitMix64, alpha_star, conv_diff_2d

pytestmark = pytest.mark.gpu
BAND = {FP64: 0.05, FP32: 0.10, BF16: 0.25}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2512_21164_gb300 import build
    build.build()


def _systems():
    out = []
    for i, (nx, ny) in enumerate([(32, 32), (24, 20), (16, 16), (40, 8)]):
        p, _ = conv_diff_2d(nx, 400 + i, ny=ny)
        out.append((p, 2.0 * alpha_star(p)))
    return out


@pytest.mark.parametrize("prec", [FP64, FP32, BF16])
@pytest.mark.parametrize("group", [0, 1, 4])  # 0: tuned group sizes
@pytest.mark.parametrize("hres", [None, 0])
def test_batched_matches_oracle(prec, group, hres):
    """hres None: the default options, under which FP32 and BF16 units take
    the SM-resident H-solve (p of a block's rows in shared memory); 0: the
    streaming H-solve.  The 40 x 8 system admits resident groups of at most
    8 blocks, so with tuned sizes the larger groups may not take its units."""
    import torch
    nrhs = 2
    systems = _systems()
    g = SplitMix64(77)
    handles, bs, xs, alphas, rhs = [], [], [], [], []
    for p, a in systems:
        orc = O.Oracle(p)
        bb = np.concatenate([orc.rhs(g.uniform_array(p.nvec)) for _ in range(nrhs)])
        rhs.append(bb)
        handles.append(G.Gadi.from_problem(p))
        bs.append(dev64(bb))
        xs.append(torch.zeros(nrhs * p.nvec, dtype=torch.float64, device="cuda"))
        alphas.append(a)
    tol_in = 1e-2 if prec == BF16 else 1e-3
    kw = {} if hres is None else dict(h_resident=hres)
    st, stats = G.solve_batched(handles, nrhs, bs, xs, alphas, 1.0, prec, 1e-10, 3000,
                                tol_h=tol_in, tol_s=tol_in, batch_group=group, **kw)
    assert st == G.OK, G.status_str(st)
    resident = hres is None and prec != FP64
    for s, (p, a) in enumerate(systems):
        orc = O.Oracle(p)
        xg_all = xs[s].cpu().numpy()
        for j in range(nrhs):
            b = rhs[s][j * p.nvec:(j + 1) * p.nvec]
            xg = xg_all[j * p.nvec:(j + 1) * p.nvec]
            u = stats[s * nrhs + j]
            _, so = orc.gadi(b, a, 1.0, prec, tol=1e-10, maxit=3000, tol_h=tol_in, tol_s=tol_in,
                             s_pointwise=True)
            assert so["status"] == "OK" and u["status"] == G.OK
            assert abs(u["outer_its"] - so["outer_its"]) <= max(2, BAND[prec] * so["outer_its"])
            rel = np.linalg.norm(b - orc.apply(O.OP_A, xg)) / np.linalg.norm(b)
            assert rel <= 1e-10
            assert u["seconds"] > 0
            assert u["blocks"] == group if group > 0 else 1 <= u["blocks"] <= 64
            assert u["h_resident"] == (1 if resident else 0)
            if resident:
                assert u["blocks"] <= p.ny
    for h in handles:
        h.close()


def test_batched_rejects_other_classes():
    import torch
    from workloads import conv_diff_3d
    p, _ = conv_diff_3d(4, 5)
    with G.Gadi.from_problem(p) as H:
        b = torch.zeros(p.nvec, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        st, _ = G.solve_batched([H], 1, [b], [x], [1.0], check=False)
    assert st == G.ERR_UNSUPPORTED


@pytest.mark.parametrize("prec", [FP32, BF16])
def test_batched_double_fp64_residual_matches_single(prec):
    """The batched kernel with the residual in double-FP64 (u_r ~ u^2): every
    unit converges and its iterate satisfies the tolerance by the oracle's
    double-FP64 residual, with outer iterations in the band of the single
    double-FP64 solve of the same system."""
    import torch
    nrhs = 2
    systems = _systems()[:3]
    g = SplitMix64(78)
    handles, bs, xs, alphas, rhs = [], [], [], [], []
    for p, a in systems:
        orc = O.Oracle(p)
        bb = np.concatenate([orc.rhs(g.uniform_array(p.nvec)) for _ in range(nrhs)])
        rhs.append(bb)
        handles.append(G.Gadi.from_problem(p))
        bs.append(dev64(bb))
        xs.append(torch.zeros(nrhs * p.nvec, dtype=torch.float64, device="cuda"))
        alphas.append(a)
    tol_in = 1e-2 if prec == BF16 else 1e-3
    st, stats = G.solve_batched(handles, nrhs, bs, xs, alphas, 1.0, prec, 1e-11, 3000,
                                tol_h=tol_in, tol_s=tol_in, batch_group=2, u_r=G.FP64X2)
    assert st == G.OK, G.status_str(st)
    for s, (p, a) in enumerate(systems):
        orc = O.Oracle(p)
        for j in range(nrhs):
            b = rhs[s][j * p.nvec:(j + 1) * p.nvec]
            xg = xs[s].cpu().numpy()[j * p.nvec:(j + 1) * p.nvec]
            _, rh, rl, _, _ = orc.residual_dd(FP64, b, xg)
            assert np.linalg.norm(rh) / np.linalg.norm(b) <= 1e-11
            x1 = torch.zeros(p.nvec, dtype=torch.float64, device="cuda")
            st1, s1 = handles[s].solve(dev64(b), x1, a, 1.0, prec, 1e-11, 3000, tol_h=tol_in, tol_s=tol_in,
                                       u_r=G.FP64X2)
            assert st1 == G.OK
            u = stats[s * nrhs + j]
            assert abs(u["outer_its"] - s1["outer_its"]) <= max(2, BAND[prec] * s1["outer_its"])
    for h in handles:
        h.close()


@pytest.mark.parametrize("interleave", [1, 0])
@pytest.mark.parametrize("group", [0, 3])
def test_batched_four_rhs_interleaved_matches_oracle(interleave, group):
    """Four right-hand sides per system, FP32 inner solves: interleaved as
    [n][4] in one unit (each right-hand side with its own scalars, stopping
    and outer iteration) or one unit each -- every right-hand side must reach
    the oracle's outcome for it, within the outer-iteration band.  One system
    gets a right-hand side of zeros (solved at x_0 = 0) and one a right-hand
    side of another shape and scale, so the units run with some right-hand
    sides frozen while others go on."""
    import torch
    nrhs = 4
    systems = _systems()
    g = SplitMix64(78)
    handles, bs, xs, alphas, rhs = [], [], [], [], []
    for si, (p, a) in enumerate(systems):
        orc = O.Oracle(p)
        cols = [orc.rhs(g.uniform_array(p.nvec)) for _ in range(nrhs)]
        if si == 0:
            cols[2] = np.zeros(p.nvec)
        if si == 1:
            cols[1] = cols[1] * 1e3 + orc.rhs(np.sin(np.arange(p.nvec) * 0.7))
        bb = np.concatenate(cols)
        rhs.append(bb)
        handles.append(G.Gadi.from_problem(p))
        bs.append(dev64(bb))
        xs.append(torch.zeros(nrhs * p.nvec, dtype=torch.float64, device="cuda"))
        alphas.append(a)
    st, stats = G.solve_batched(handles, nrhs, bs, xs, alphas, 1.0, FP32, 1e-10, 3000, tol_h=1e-3, tol_s=1e-3,
                                batch_group=group, batch_interleave=interleave)
    assert st == G.OK, G.status_str(st)
    for s, (p, a) in enumerate(systems):
        orc = O.Oracle(p)
        xg_all = xs[s].cpu().numpy()
        for j in range(nrhs):
            b = rhs[s][j * p.nvec:(j + 1) * p.nvec]
            xg = xg_all[j * p.nvec:(j + 1) * p.nvec]
            u = stats[s * nrhs + j]
            _, so = orc.gadi(b, a, 1.0, FP32, tol=1e-10, maxit=3000, tol_h=1e-3, tol_s=1e-3)
            assert so["status"] == "OK" and u["status"] == G.OK, (s, j, so["status"], u["status"])
            assert abs(u["outer_its"] - so["outer_its"]) <= max(2, BAND[FP32] * so["outer_its"]), \
                (s, j, u["outer_its"], so["outer_its"])
            if not np.any(b):
                assert u["outer_its"] == 0 and not np.any(xg)
                continue
            rel = np.linalg.norm(b - orc.apply(O.OP_A, xg)) / np.linalg.norm(b)
            assert rel <= 1e-10, (s, j, rel)
    for h in handles:
        h.close()
