"""Whole solves (Algorithm 1) on the GPU against the CPU oracle.

Acceptance: the GPU reaches the oracle's outcome (relative residual and
normwise backward error <= 1e-10 when the oracle does), its forward error is
within 10x the oracle's, and its outer iteration count is within +-5% (FP64
inner), +-10% (FP32) or +-25% (BF16) of the oracle's.  Also: the 64 x 64
plain-FP64 run of 500 iterations, host-pointer and device-pointer calls
agreeing bit for bit, run-to-run determinism, argument validation and the
||A||_2 estimate.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_2512_21164_gb300 as G
from helpers import BF16, FP32, FP64, dev64
from workloads import alpha_star, complex_rd, config1, conv_diff_2d, conv_diff_3d, random_csr

pytestmark = pytest.mark.gpu

BAND = {FP64: 0.05, FP32: 0.10, BF16: 0.25}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2512_21164_gb300 import build
    build.build()


def _tols(prec):
    return (1e-2, 1e-2) if prec == BF16 else (1e-3, 1e-3)


def _gpu_solve(p, b, alpha, omega, prec, tol, maxit, **kw):
    import torch
    x = torch.zeros(p.nvec, dtype=torch.float64, device="cuda")
    hist = np.zeros(maxit + 2)
    th, ts = _tols(prec)
    opts = dict(tol_h=th, tol_s=ts)
    opts.update(kw)
    with G.Gadi.from_problem(p) as H:
        st, stats = H.solve(dev64(b), x, alpha, omega, prec, tol, maxit, hist=hist, **opts)
    return st, stats, x.cpu().numpy(), hist[:stats["outer_its"] + 1]


def _cases():
    out = []
    for prec in (FP64, FP32, BF16):
        p, xt = conv_diff_2d(48, 201, ny=40)
        out.append(("2d", p, xt, 2 * alpha_star(p), 1.0, prec))
        p, xt = conv_diff_3d(12, 202)
        out.append(("3d", p, xt, 2 * alpha_star(p), 1.0, prec))
        p, xt = complex_rd(24, 203)
        out.append(("cplx", p, xt, alpha_star(p), 1.0, prec))
        p, xt = random_csr(400, 204)
        out.append(("csr", p, xt, 1.0, 1.0, prec))
    return out


@pytest.mark.parametrize("name,p,xt,alpha,omega,prec", _cases(),
                         ids=[f"{c[0]}-{c[5]}" for c in _cases()])
def test_solve_matches_oracle(name, p, xt, alpha, omega, prec):
    orc = O.Oracle(p)
    b = orc.rhs(xt)
    th, ts = _tols(prec)
    xo, so = orc.gadi(b, alpha, omega, prec, tol=1e-10, maxit=3000, tol_h=th, tol_s=ts,
                      s_pointwise=True)
    st, sg, xg, hg = _gpu_solve(p, b, alpha, omega, prec, 1e-10, 3000)
    assert so["status"] == "OK"
    assert st == G.OK, G.status_str(st)
    assert abs(sg["outer_its"] - so["outer_its"]) <= max(2, BAND[prec] * so["outer_its"]), \
        (sg["outer_its"], so["outer_its"])
    # FP64 residual and backward error of the GPU iterate, by the oracle
    r = b - orc.apply(O.OP_A, xg)
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert rel <= 1e-10 and abs(rel - sg["relres"]) <= 1e-3 * rel
    Anorm = O.norm2_power(lambda v: orc.apply(O.OP_A, v),
                          lambda v: orc.apply(O.OP_M, v) - orc.apply(O.OP_N, v), p.nvec, iters=30)
    assert O.backward_error(np.linalg.norm(r), Anorm, xg, b) <= 1e-10
    fe_g = np.linalg.norm(xg - xt) / np.linalg.norm(xt)
    fe_o = np.linalg.norm(xo - xt) / np.linalg.norm(xt)
    assert fe_g <= 10 * fe_o + 1e-14, (fe_g, fe_o)
    # the relres histories follow the same trajectory
    k = min(len(hg), len(so["history"]))
    ratio = np.abs(np.log10(hg[1:k] / so["history"][1:k]))
    assert np.median(ratio) < 0.3


def test_config1_plain_fp64_500_iterations():
    """64 x 64, beta=(10,10), alpha=0.5, omega=1, maxit 500, plain FP64: the
    run ends at the cap (relres ~6e-9) on both sides."""
    p, xt, c = config1()
    orc = O.Oracle(p)
    b = orc.rhs(xt)
    xo, so = orc.gadi(b, c["alpha"], c["omega"], FP64, tol=c["tol"], maxit=c["maxit"])
    st, sg, xg, hg = _gpu_solve(p, b, c["alpha"], c["omega"], FP64, c["tol"], c["maxit"])
    assert so["status"] == "NOT_CONVERGED" and st == G.NOT_CONVERGED
    assert sg["outer_its"] == so["outer_its"] == 500
    assert abs(math.log10(sg["relres"] / so["relres"])) < 0.05
    assert np.allclose(hg, so["history"], rtol=1e-2, atol=0)
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)


def test_host_and_device_pointers_agree_and_deterministic():
    import torch
    p, xt = conv_diff_2d(40, 205)
    b = O.Oracle(p).rhs(xt)
    a = alpha_star(p) * 2
    with G.Gadi.from_problem(p) as H:
        xh = np.zeros(p.nvec)
        st1, s1 = H.solve(b, xh, a, 1.0, FP32, 1e-10, 2000)
        xd = torch.zeros(p.nvec, dtype=torch.float64, device="cuda")
        st2, s2 = H.solve(dev64(b), xd, a, 1.0, FP32, 1e-10, 2000)
        xd2 = torch.zeros_like(xd)
        st3, s3 = H.solve(dev64(b), xd2, a, 1.0, FP32, 1e-10, 2000)
    assert st1 == st2 == st3 == G.OK
    assert np.array_equal(xh, xd.cpu().numpy())
    assert torch.equal(xd, xd2)
    assert s1["outer_its"] == s2["outer_its"] == s3["outer_its"]
    assert s1["inner_its_h"] == s2["inner_its_h"]


def test_argument_validation_and_edge_cases():
    import torch
    p, xt = conv_diff_2d(16, 206)
    b = O.Oracle(p).rhs(xt)
    with G.Gadi.from_problem(p) as H:
        x = np.zeros(p.nvec)
        for kw in [dict(alpha=0.0), dict(alpha=-1.0), dict(omega=2.0), dict(omega=-0.1)]:
            args = dict(alpha=0.5, omega=1.0)
            args.update(kw)
            st, _ = H.solve(b, x, args["alpha"], args["omega"], FP32, 1e-10, 10, check=False)
            assert st == G.ERR_INVALID
        bn = b.copy()
        bn[3] = np.nan
        st, _ = H.solve(bn, x, 0.5, 1.0, FP32, 1e-10, 10, check=False)
        assert st == G.ERR_NONFINITE
        st, _ = H.solve(dev64(bn), torch.zeros(p.nvec, dtype=torch.float64, device="cuda"), 0.5,
                        1.0, FP32, 1e-10, 10, check=False)
        assert st == G.ERR_NONFINITE
        assert np.all(x == 0)
        # maxit = 0: one residual, no update
        x0 = np.full(p.nvec, 0.25)
        st, s = H.solve(b, x0, 0.5, 1.0, FP32, 1e-10, 0)
        assert st == G.NOT_CONVERGED and s["outer_its"] == 0 and np.all(x0 == 0.25)
        # b = 0 with x0 = 0: already solved
        z = np.zeros(p.nvec)
        st, s = H.solve(np.zeros(p.nvec), z, 0.5, 1.0, BF16, 1e-10, 10)
        assert st == G.OK and s["outer_its"] == 0 and np.all(z == 0)
    with pytest.raises(G.GadiError):
        G.Gadi(G.STENCIL_2D5, 0, 5)
    with pytest.raises(G.GadiError):
        G.Gadi(G.CSR, rowptr=[0, 1], col=[3], val=[1.0])


def test_norm2_estimate():
    p, xt = conv_diff_2d(20, 207, ny=17)
    orc = O.Oracle(p)
    A = orc.dense(O.OP_A)
    with G.Gadi.from_problem(p) as H:
        est = H.norm2(200)
    true = np.linalg.norm(A, 2)
    assert 0.999 * true <= est <= true * (1 + 1e-10)


def test_alpha_restarts_recover_from_stagnation():
    """Sec. 4.3 (a larger alpha after stagnation): a BF16 run with a too-small alpha stagnates; with
    restarts, alpha is doubled from the last iterate until it converges."""
    p, xt = conv_diff_2d(48, 9)
    orc = O.Oracle(p)
    b = orc.rhs(xt)
    a = alpha_star(p) / 16
    import torch
    with G.Gadi.from_problem(p) as H:
        x = torch.zeros(p.nvec, dtype=torch.float64, device="cuda")
        st, s = H.solve(dev64(b), x, a, 1.0, BF16, 1e-10, 5000, outer_stag_window=5)
        assert st == G.STAGNATED
        x.zero_()
        st, s = H.solve(dev64(b), x, a, 1.0, BF16, 1e-10, 5000, outer_stag_window=5, alpha_restarts=10)
    assert st == G.OK, G.status_str(st)
    assert s["restarts"] >= 1 and s["alpha"] > a
    xg = x.cpu().numpy()
    rel = np.linalg.norm(b - orc.apply(O.OP_A, xg)) / np.linalg.norm(b)
    assert rel <= 1e-10 and abs(rel - s["relres"]) <= 1e-2 * rel


def test_barrier_wait_runs_out_and_device_stays_usable():
    """A grid barrier that one block never reaches: the others' bounded waits
    run out, the kernel unwinds and the host reads GADI_ERR_TIMEOUT; a solve
    afterwards still works."""
    assert G.selftest_barrier(64, 50.0) == G.ERR_TIMEOUT
    p, xt = conv_diff_2d(24, 210)
    b = O.Oracle(p).rhs(xt)
    with G.Gadi.from_problem(p) as H:
        x = np.zeros(p.nvec)
        st, s = H.solve(b, x, 2 * alpha_star(p), 1.0, FP32, 1e-10, 2000)
    assert st == G.OK


@pytest.mark.parametrize("prec", [FP32, BF16])
@pytest.mark.parametrize("max_blocks", [16, 40])
def test_resident_h_solve_matches_streaming_and_oracle(prec, max_blocks):
    """The 2D real class with p of CG on H held in shared memory (2-3 rows per
    block, and exactly one row per block) against the streaming form and the
    oracle: same arithmetic, only the order of the grid-wide sums differs."""
    p, xt = conv_diff_2d(48, 201, ny=40)
    orc = O.Oracle(p)
    b = orc.rhs(xt)
    alpha = 2 * alpha_star(p)
    th, ts = _tols(prec)
    xo, so = orc.gadi(b, alpha, 1.0, prec, tol=1e-10, maxit=3000, tol_h=th, tol_s=ts)
    res, xs = {}, {}
    for hr in (2, 1, 0):
        st, sg, xg, hg = _gpu_solve(p, b, alpha, 1.0, prec, 1e-10, 3000, max_blocks=max_blocks,
                                    h_resident=hr, s_resident=0)
        assert st == G.OK, G.status_str(st)
        assert sg["h_resident"] == hr and sg["blocks"] == max_blocks
        rel = np.linalg.norm(b - orc.apply(O.OP_A, xg)) / np.linalg.norm(b)
        assert rel <= 1e-10
        assert abs(sg["outer_its"] - so["outer_its"]) <= max(2, BAND[prec] * so["outer_its"])
        res[hr], xs[hr] = sg, xg
    assert abs(res[1]["outer_its"] - res[0]["outer_its"]) <= max(2, BAND[prec] * res[0]["outer_its"])
    assert abs(res[1]["inner_its_h"] - res[0]["inner_its_h"]) <= 0.1 * res[0]["inner_its_h"] + 2
    # z and r in tensor memory: the same operations in the same order as 1
    assert np.array_equal(xs[2], xs[1])
    for key in ("outer_its", "inner_its_h", "inner_its_s", "relres"):
        assert res[2][key] == res[1][key]


def _tm_slots(nx, ny, prec, blocks, threads=512):
    """Slots per thread the tensor-memory H-solve needs (16 available)."""
    nxw = nx // (4 if prec == FP32 else 8)
    worst = 0
    for bi in range(blocks):
        R = (bi + 1) * ny // blocks - bi * ny // blocks
        need = -(-nxw // threads) * R if nxw >= threads else -(-R // (threads // nxw))
        worst = max(worst, need)
    return worst


@pytest.mark.parametrize("prec", [FP32, BF16])
@pytest.mark.parametrize("nx,ny,blocks", [(2560, 200, 16), (8, 400, 16), (4096, 160, 16), (2048, 304, 152)])
def test_tmem_h_solve_same_bits_as_shared_memory_form(prec, nx, ny, blocks):
    """h_resident = 2 keeps z and r of CG on H in tensor memory when each
    thread's chunks fit 16 slots, else falls back to 1: either way the result
    has the same bits as h_resident = 1 (two column passes, row parts of a
    narrow grid, a shape past the slot limit in FP32)."""
    import torch
    p, xt = conv_diff_2d(nx, 212, ny=ny)
    a0 = alpha_star(p)
    out = {}
    with G.Gadi.from_problem(p) as H:
        xtd = torch.from_numpy(np.ascontiguousarray(xt)).cuda()
        b = torch.zeros_like(xtd)
        H.apply(G.OP_A, xtd, b)
        th, ts = _tols(prec)
        for hr in (2, 1):
            x = torch.zeros_like(b)
            st, s = H.solve(b, x, 4 * a0, 0.0, prec, 1e-12, 4, tol_h=th, tol_s=ts, max_blocks=blocks,
                            h_resident=hr, s_resident=0, check=False)
            assert st in (G.OK, G.NOT_CONVERGED), G.status_str(st)
            out[hr] = (s, x.cpu().numpy())
    want = 2 if _tm_slots(nx, ny, prec, blocks) <= 16 else 1
    assert out[2][0]["h_resident"] == want and out[1][0]["h_resident"] == 1
    assert np.array_equal(out[2][1], out[1][1])
    for key in ("outer_its", "inner_its_h", "inner_its_s", "relres"):
        assert out[2][0][key] == out[1][0][key]


@pytest.mark.parametrize("prec", [FP32, BF16])
@pytest.mark.parametrize("nx,ny,blocks", [(48, 40, 16), (48, 32, 16), (48, 16, 16), (8, 400, 16),
                                          (2560, 200, 16), (2560, 120, 16)])
def test_resident_cgnr_matches_streaming(prec, nx, ny, blocks):
    """CGNR on S with p in shared memory and t, y in tensor memory
    (s_resident = 1, taken with the tensor-memory H-solve when every block
    owns two rows or more; 2560 x 200 FP32 needs more than 16 slots and
    takes neither, 2560 x 120 FP32 fills all 16 with two column passes)
    against
    the streaming S-solve (s_resident = 0): both reach 1e-10, outer
    iterations within the precision's band, and the small grids against the
    oracle."""
    import torch
    p, xt = conv_diff_2d(nx, 213, ny=ny)
    a0 = alpha_star(p)
    th, ts = _tols(prec)
    out = {}
    with G.Gadi.from_problem(p) as H:
        xtd = torch.from_numpy(np.ascontiguousarray(xt)).cuda()
        b = torch.zeros_like(xtd)
        H.apply(G.OP_A, xtd, b)
        r = torch.zeros_like(b)
        for sr in (1, 0):
            x = torch.zeros_like(b)
            st, s = H.solve(b, x, 2 * a0, 1.0, prec, 1e-10, 4000, tol_h=th, tol_s=ts, max_blocks=blocks,
                            h_resident=2, s_resident=sr)
            assert st == G.OK, G.status_str(st)
            H.apply(G.OP_A, x, r)
            rel = float(torch.linalg.norm(b - r) / torch.linalg.norm(b))
            assert rel <= 1e-10
            out[sr] = (s, x.cpu().numpy())
    tm = _tm_slots(nx, ny, prec, blocks) <= 16
    want = 1 if tm and ny // blocks >= 2 else 0
    assert out[1][0]["s_resident"] == want and out[0][0]["s_resident"] == 0
    assert out[1][0]["h_resident"] == (2 if tm else 1)
    o1, o0 = out[1][0]["outer_its"], out[0][0]["outer_its"]
    assert abs(o1 - o0) <= max(2, BAND[prec] * o0)
    if nx * ny <= 4096:
        orc = O.Oracle(p)
        xo, so = orc.gadi(orc.rhs(xt), 2 * a0, 1.0, prec, tol=1e-10, maxit=4000, tol_h=th, tol_s=ts)
        assert abs(o1 - so["outer_its"]) <= max(2, BAND[prec] * so["outer_its"])
        fo = np.linalg.norm(xo - xt) / np.linalg.norm(xt)
        f1 = np.linalg.norm(out[1][1] - xt) / np.linalg.norm(xt)
        assert f1 <= 10 * fo + 1e-12


def test_resident_option_validated():
    p, xt = conv_diff_2d(16, 206)
    b = O.Oracle(p).rhs(xt)
    with G.Gadi.from_problem(p) as H:
        for bad in (3, -1):
            st, _ = H.solve(b, np.zeros(p.nvec), 0.5, 1.0, FP32, 1e-10, 10, h_resident=bad, check=False)
            assert st == G.ERR_INVALID
        for bad in (2, -1):
            st, _ = H.solve(b, np.zeros(p.nvec), 0.5, 1.0, FP32, 1e-10, 10, s_resident=bad, check=False)
            assert st == G.ERR_INVALID


@pytest.mark.parametrize("name,prec", [("2d", FP32), ("3d", BF16), ("cplx", FP32), ("csr", FP64)])
def test_double_fp64_residual_solve_matches_oracle(name, prec):
    """Algorithm 1 with u_r = double-FP64 on the GPU against the oracle's."""
    p, xt, alpha, omega = {
        "2d": lambda: (*conv_diff_2d(48, 211, ny=40), None, 1.0),
        "3d": lambda: (*conv_diff_3d(12, 212), None, 1.0),
        "cplx": lambda: (*complex_rd(24, 213), None, 1.0),
        "csr": lambda: (*random_csr(400, 214), 1.0, 1.0),
    }[name]()
    if alpha is None:
        alpha = (1.0 if p.kind == 2 else 2.0) * alpha_star(p)
    orc = O.Oracle(p)
    b = orc.rhs(xt)
    th, ts = _tols(prec)
    xo, so = orc.gadi(b, alpha, omega, prec, tol=1e-12, maxit=3000, tol_h=th, tol_s=ts, s_pointwise=True,
                      residual_dd=True)
    st, sg, xg, hg = _gpu_solve(p, b, alpha, omega, prec, 1e-12, 3000, u_r=G.FP64X2)
    assert so["status"] == "OK" and st == G.OK, G.status_str(st)
    assert abs(sg["outer_its"] - so["outer_its"]) <= max(2, BAND[prec] * so["outer_its"])
    _, rh, rl, _, _ = orc.residual_dd(FP64, b, xg)
    assert np.linalg.norm(rh) / np.linalg.norm(b) <= 1e-12


def test_double_fp64_residual_limits_forward_error_gpu():
    """Sec. 3 on the GPU: run to stagnation with FP32 inner solves; with
    u_r = double-FP64 the forward error reaches about u, with u_r = FP64 it
    stays several times larger (it grows with kappa(A) u_r)."""
    from test_oracle_residual_dd import forward_error_case, reference_solution
    p, xt, alpha = forward_error_case()
    b = O.Oracle(p).rhs(xt)
    xref = reference_solution(p, b)
    fe = {}
    for ur in (G.FP64, G.FP64X2):
        st, s, xg, _ = _gpu_solve(p, b, alpha, 0.0, FP32, 0.0, 20000, u_r=ur, tol_h=1e-4, tol_s=1e-4,
                                  outer_stag_window=200)
        assert st == G.STAGNATED, G.status_str(st)
        fe[ur] = np.linalg.norm(xg - xref) / np.linalg.norm(xref)
    assert fe[G.FP64X2] <= 4 * 2.0 ** -53, fe
    assert fe[G.FP64] >= 4 * fe[G.FP64X2], fe


@pytest.mark.parametrize("prec", [FP64, FP32, BF16])
def test_paper_2d_instance_matches_oracle(prec):
    """Sec. 5.2's own instance (reaction term on the diagonal, strong
    convection) at 48 x 48 against the oracle."""
    from workloads import paper_cdr_2d
    p, xt = paper_cdr_2d(48)
    orc = O.Oracle(p)
    b = orc.rhs(xt)
    a = 4 * alpha_star(p)
    th, ts = _tols(prec)
    xo, so = orc.gadi(b, a, 0.0, prec, tol=1e-10, maxit=3000, tol_h=th, tol_s=ts)
    st, sg, xg, hg = _gpu_solve(p, b, a, 0.0, prec, 1e-10, 3000)
    assert so["status"] == "OK" and st == G.OK, G.status_str(st)
    assert abs(sg["outer_its"] - so["outer_its"]) <= max(2, BAND[prec] * so["outer_its"])
    assert np.linalg.norm(b - orc.apply(O.OP_A, xg)) / np.linalg.norm(b) <= 1e-10


@pytest.mark.parametrize("prec", [FP64, FP32, BF16])
def test_paper_complex_instance_matches_oracle(prec):
    """Sec. 5.4's own instance (random per-point potential) at 48 x 48 against
    the oracle: pointwise S-solve with the per-point diagonal."""
    from workloads import paper_complex_rd
    p, xt = paper_complex_rd(48)
    orc = O.Oracle(p)
    b = orc.rhs(xt)
    a = 64 * alpha_star(p)
    th, ts = _tols(prec)
    xo, so = orc.gadi(b, a, 1.0, prec, tol=1e-10, maxit=3000, tol_h=th, tol_s=ts, s_pointwise=True)
    st, sg, xg, hg = _gpu_solve(p, b, a, 1.0, prec, 1e-10, 3000)
    assert so["status"] == "OK" and st == G.OK, G.status_str(st)
    assert abs(sg["outer_its"] - so["outer_its"]) <= max(2, BAND[prec] * so["outer_its"])
    assert np.linalg.norm(b - orc.apply(O.OP_A, xg)) / np.linalg.norm(b) <= 1e-10


def test_headline_geometry_solve_matches_oracle():
    """The 2048^2 benchmark's kernel configuration on a grid the oracle
    solves in about a minute: FP32 inner, omega = 0, inner tolerances 1e-3,
    2048 x 224 on 16 blocks -- 14 rows per block and one column pass, as each
    of the benchmark's 152 blocks has on 2048^2 -- so the H-solve keeps p in
    shared memory and z, r in tensor memory (14 of 16 slots) and CGNR on S
    runs resident.  alpha = 2 alpha* of this grid (about 1200 outer
    iterations; 8 alpha* needs about 4500 on this narrower grid).  The
    oracle runs in its all-core build (the same arithmetic, its sums split by
    thread).  Against it: outer iterations within +-10 %, relres and backward
    error <= 1e-10, forward error within 10x, and the opt-in backward error
    of gadi_stats."""
    p, xt = conv_diff_2d(2048, 2, ny=224)
    orc = O.Oracle(p)
    b = orc.rhs(xt)
    alpha = 2 * alpha_star(p)
    omp = O.Oracle(p, omp=True) if O.has_openmp() else orc
    xo, so = omp.gadi(b, alpha, 0.0, FP32, tol=1e-10, maxit=20000, tol_h=1e-3, tol_s=1e-3)
    st, sg, xg, hg = _gpu_solve(p, b, alpha, 0.0, FP32, 1e-10, 20000, max_blocks=16, backward_err=50)
    assert so["status"] == "OK" and st == G.OK, (so["status"], G.status_str(st))
    assert (sg["blocks"], sg["h_resident"], sg["s_resident"]) == (16, 2, 1), sg
    assert abs(sg["outer_its"] - so["outer_its"]) <= max(2, 0.10 * so["outer_its"]), \
        (sg["outer_its"], so["outer_its"])
    r = b - orc.apply(O.OP_A, xg)
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert rel <= 1e-10 and abs(rel - sg["relres"]) <= 1e-3 * rel
    Anorm = O.norm2_power(lambda v: orc.apply(O.OP_A, v),
                          lambda v: orc.apply(O.OP_M, v) - orc.apply(O.OP_N, v), p.nvec, iters=50)
    be = O.backward_error(np.linalg.norm(r), Anorm, xg, b)
    assert be <= 1e-10
    assert abs(sg["backward_err"] - be) <= 1e-2 * be, (sg["backward_err"], be)
    fe_g = np.linalg.norm(xg - xt) / np.linalg.norm(xt)
    fe_o = np.linalg.norm(xo - xt) / np.linalg.norm(xt)
    assert fe_g <= 10 * fe_o + 1e-14, (fe_g, fe_o)


@pytest.mark.parametrize("prec", [FP64, FP32, BF16])
@pytest.mark.parametrize("blocks", [4, 0])
def test_3d_plane_ring_solve_matches_oracle(prec, blocks):
    """The 3D FP32 inner phases with 16-byte rows march a block's tile of y
    rows through z together, staging planes in shared memory (BF16 and FP64
    take the register ring on the same shapes).  On 24 x 40 x 64
    (three y-tiles, the last one partial, one partial strip) with 4 blocks
    every block marches 48 planes and crosses from one column to the next;
    with the default grid (one block per SM) most blocks take one to two
    planes.  Against the oracle: outer iterations within the band, relres
    <= 1e-10 by the oracle's residual, forward error within 10x."""
    from workloads import K_3D7, Problem, SplitMix64
    p = Problem(K_3D7, 24, 40, 64, 1.0 / 25, (10.0, 20.0, 30.0))
    xt = SplitMix64(219).uniform_array(p.nvec)
    orc = O.Oracle(p)
    b = orc.rhs(xt)
    a = 2 * alpha_star(p)
    th, ts = _tols(prec)
    xo, so = orc.gadi(b, a, 1.0, prec, tol=1e-10, maxit=3000, tol_h=th, tol_s=ts, s_pointwise=True)
    kw = dict(max_blocks=blocks) if blocks else {}
    st, sg, xg, hg = _gpu_solve(p, b, a, 1.0, prec, 1e-10, 3000, **kw)
    assert so["status"] == "OK" and st == G.OK, G.status_str(st)
    if blocks:
        assert sg["blocks"] == blocks
    assert abs(sg["outer_its"] - so["outer_its"]) <= max(2, BAND[prec] * so["outer_its"]), \
        (sg["outer_its"], so["outer_its"])
    assert np.linalg.norm(b - orc.apply(O.OP_A, xg)) / np.linalg.norm(b) <= 1e-10
    fe_g = np.linalg.norm(xg - xt) / np.linalg.norm(xt)
    fe_o = np.linalg.norm(xo - xt) / np.linalg.norm(xt)
    assert fe_g <= 10 * fe_o + 1e-14, (fe_g, fe_o)


@pytest.mark.parametrize("prec", [FP64, FP32, BF16])
def test_backward_err_stat_matches_oracle(prec):
    """gadi_stats.backward_err (opt-in) is eq. (3.2) of the returned x, host
    and device vectors alike; off by default (-1)."""
    import torch
    p, xt = conv_diff_2d(40, 211, ny=36)
    orc = O.Oracle(p)
    b = orc.rhs(xt)
    a = 2 * alpha_star(p)
    with G.Gadi.from_problem(p) as H:
        xd = torch.zeros(p.nvec, dtype=torch.float64, device="cuda")
        st, s = H.solve(dev64(b), xd, a, 1.0, prec, 1e-8, 2000, backward_err=400)
        xh = np.zeros(p.nvec)
        st2, s2 = H.solve(b, xh, a, 1.0, prec, 1e-8, 2000, backward_err=400)
        _, s3 = H.solve(b, np.zeros(p.nvec), a, 1.0, prec, 1e-8, 2000)
    assert st == st2 == G.OK and s3["backward_err"] == -1.0
    xg = xd.cpu().numpy()
    # ||A||_2 exactly (dense SVD): power iteration gives a lower bound of it,
    # so the reported backward error is at or just above the exact one
    Anorm = np.linalg.norm(orc.dense(O.OP_A), 2)
    be = O.backward_error(np.linalg.norm(b - orc.apply(O.OP_A, xg)), Anorm, xg, b)
    assert be * (1 - 1e-12) <= s["backward_err"] <= be * (1 + 5e-3), (s["backward_err"], be)
    assert abs(s2["backward_err"] - s["backward_err"]) <= 1e-12 * be


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_diverged_rule_matches_oracle(prec):
    """A = -(1 + 1/4) I (CSR): relres_k = 9^k exactly in closed form, so both
    sides must report DIVERGED at the first k with relres > 1e6 (k = 7)."""
    from workloads import K_CSR, Problem
    n = 4
    p = Problem(K_CSR, n, rowptr=np.arange(n + 1, dtype=np.int32), col=np.arange(n, dtype=np.int32),
                val=np.full(n, -1.25))
    orc = O.Oracle(p)
    b = np.array([1.0, -2.0, 0.5, 3.0])
    _, so = orc.gadi(b, 1.0, 0.0, prec, tol=1e-10, maxit=50, outer_stag_window=0)
    st, sg, xg, hg = _gpu_solve(p, b, 1.0, 0.0, prec, 1e-10, 50, outer_stag_window=0)
    assert so["status"] == "DIVERGED" and st == G.DIVERGED
    assert sg["outer_its"] == so["outer_its"] == 7
    # FP32 inner solves round r_s: the closed form then holds to u_s per step
    assert np.allclose(hg, 9.0 ** np.arange(8), rtol=1e-9 if prec == FP64 else 1e-5)


@pytest.mark.parametrize("prec", [FP64, FP32, BF16])
def test_stencil_matrix_as_csr_matches_oracle_and_stencil(prec):
    """The benchmark's matrix class (2D convection-diffusion, beta drawn by
    seed 2) assembled as CSR and solved by the CSR kernels: against the
    oracle's solve of the CSR it assembles from its own coefficients, and
    against the stencil kernels on the same system (alpha = 8 alpha*,
    omega = 0, inner tolerances of the precision)."""
    from test_csr_assembly import oracle_csr
    from workloads import K_CSR, Problem
    p, xt = conv_diff_2d(64, 2, ny=48)
    rp, cl, vl = G.stencil_csr(p)
    pc = Problem(K_CSR, p.npoints, rowptr=rp, col=cl, val=vl)
    orp, ocl, ovl = oracle_csr(p)
    po = Problem(K_CSR, p.npoints, rowptr=orp, col=ocl, val=ovl)
    orc = O.Oracle(po)
    b = orc.rhs(xt)
    alpha = 8 * alpha_star(p)
    th, ts = _tols(prec)
    xo, so = orc.gadi(b, alpha, 0.0, prec, tol=1e-10, maxit=20000, tol_h=th, tol_s=ts)
    st, sg, xg, _ = _gpu_solve(pc, b, alpha, 0.0, prec, 1e-10, 20000)
    st2, sg2, xg2, _ = _gpu_solve(p, b, alpha, 0.0, prec, 1e-10, 20000)
    assert so["status"] == "OK" and st == G.OK and st2 == G.OK
    band = max(2, BAND[prec] * so["outer_its"])
    assert abs(sg["outer_its"] - so["outer_its"]) <= band, (sg["outer_its"], so["outer_its"])
    assert abs(sg2["outer_its"] - sg["outer_its"]) <= band, (sg2["outer_its"], sg["outer_its"])
    for xv in (xg, xg2):
        rel = np.linalg.norm(b - orc.apply(O.OP_A, xv)) / np.linalg.norm(b)
        assert rel <= 1e-10, rel
    fe_o = np.linalg.norm(xo - xt) / np.linalg.norm(xt)
    assert np.linalg.norm(xg - xt) / np.linalg.norm(xt) <= 10 * fe_o + 1e-14


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_config3_twin_matches_oracle(prec):
    """The 512^3 benchmark's 64^3 twin (beta = (1,1,1) U[1,50] by the same
    seed, alpha = alpha*, omega = 0, the alpha and omega the 512^3 lines use)
    against the oracle (its all-core build): outer iterations in the band,
    relres and backward error <= 1e-10, forward error within 10x."""
    from workloads import config3
    p, xt = config3(64)
    orc = O.Oracle(p)
    b = orc.rhs(xt)
    alpha = alpha_star(p)
    omp = O.Oracle(p, omp=True) if O.has_openmp() else orc
    xo, so = omp.gadi(b, alpha, 0.0, prec, tol=1e-10, maxit=20000, tol_h=1e-3, tol_s=1e-3)
    st, sg, xg, _ = _gpu_solve(p, b, alpha, 0.0, prec, 1e-10, 20000, backward_err=50)
    assert so["status"] == "OK" and st == G.OK, (so["status"], G.status_str(st))
    assert abs(sg["outer_its"] - so["outer_its"]) <= max(2, BAND[prec] * so["outer_its"]), \
        (sg["outer_its"], so["outer_its"])
    r = b - orc.apply(O.OP_A, xg)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10
    assert sg["backward_err"] <= 1e-10
    fe_o = np.linalg.norm(xo - xt) / np.linalg.norm(xt)
    assert np.linalg.norm(xg - xt) / np.linalg.norm(xt) <= 10 * fe_o + 1e-14
