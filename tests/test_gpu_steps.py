"""GPU parity of each step of Algorithm 1 against the CPU oracle.

The residual step and the operator application are elementwise FP64 in the
same operation order on both sides, so they must agree bit for bit (up to the
sign of zero).  The inner solves agree up to the summation order of the dot
products; with a fixed iteration count they are compared elementwise within
a tolerance derived from u_s, and to convergence by iteration count and by
the true residual of the result.  Grids cover the 16-byte vector path, the
narrow path (odd row lengths), single rows / columns, ragged last strips,
3D and complex grids, and general CSR matrices.
"""
import numpy as np
import pytest

import oracle as O
import paper_2512_21164_gb300 as G
from helpers import BF16, FP32, FP64, PRECS, dev64, us_empty, us_to_device, us_to_host
from workloads import (K_3D7, Problem, SplitMix64, complex_rd, conv_diff_2d, conv_diff_3d, paper_complex_rd,
                       random_csr)

pytestmark = pytest.mark.gpu

CASES = {
    "2d_vec": lambda: conv_diff_2d(64, 101, ny=48),
    "2d_ragged": lambda: conv_diff_2d(37, 102, ny=5),
    "2d_row": lambda: conv_diff_2d(300, 103, ny=1),
    "2d_col": lambda: conv_diff_2d(1, 104, ny=70),
    "2d_wide": lambda: conv_diff_2d(1032, 105, ny=9),
    "2d_one": lambda: conv_diff_2d(1, 110, ny=1),
    # more rows than persistent blocks (one per SM): the H-solve keeps p in
    # shared memory (4-5 rows per block, and 1-2 rows per block)
    "2d_tall": lambda: conv_diff_2d(64, 112, ny=700),
    "2d_slab1": lambda: conv_diff_2d(40, 113, ny=170),
    # resident H-solve with fewer 16-byte chunks per row than threads (the
    # block's rows split into parts) and with more (two column passes)
    "2d_narrow_tall": lambda: conv_diff_2d(8, 116, ny=400),
    "2d_wide_tall": lambda: conv_diff_2d(2560, 117, ny=200),
    "3d_vec": lambda: conv_diff_3d(16, 106),
    "3d_ragged": lambda: (Problem(K_3D7, 7, 5, 9, 1.0 / 8, (13.0, 29.0, 41.0)),
                          SplitMix64(111).uniform_array(7 * 5 * 9)),
    "cplx_vec": lambda: complex_rd(32, 107),
    "cplx_odd": lambda: complex_rd(13, 108),
    # per-point imaginary diagonal (the random potential of Sec. 5.4)
    "cplx_pt": lambda: paper_complex_rd(32, 115),
    "csr": lambda: random_csr(300, 109),
}


def rnd(prec, a):
    if prec == FP64:
        return np.asarray(a, np.float64).copy()
    if prec == FP32:
        return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)
    return np.array([O.round_bf16(v) for v in a])


def ulp_bf16(a):
    e = np.floor(np.log2(np.maximum(np.abs(a), 2.0 ** -126)))
    return 2.0 ** (e - 7)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2512_21164_gb300 import build
    build.build()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("with_y", [False, True])
def test_residual_step_bit_exact(case, prec, with_y):
    import torch
    p, xt = CASES[case]()
    orc = O.Oracle(p)
    m = p.nvec
    g = SplitMix64(7)
    x = g.uniform_array(m) - 0.5
    b = orc.rhs(xt)
    y = rnd(prec, (g.uniform_array(m) - 0.5) * 1e-2) if with_y else None
    with G.Gadi.from_problem(p) as H:
        xo = torch.zeros(m, dtype=torch.float64, device="cuda")
        ro = torch.zeros_like(xo)
        rs = us_empty(m, prec)
        nrm = H.step_residual(prec, dev64(b), dev64(x), us_to_device(y, prec) if with_y else None,
                              xo, ro, rs)
    xo_o, r_o, rs_o, n_o = orc.residual(prec, b, x, y)
    assert np.array_equal(xo.cpu().numpy(), xo_o)
    assert np.array_equal(ro.cpu().numpy(), r_o)
    assert np.array_equal(us_to_host(rs, prec), rs_o)
    assert abs(nrm - n_o) <= 1e-12 * n_o


@pytest.mark.parametrize("case", ["2d_vec", "2d_ragged", "3d_ragged", "cplx_odd", "csr"])
def test_apply_operators(case):
    import torch
    p, xt = CASES[case]()
    orc = O.Oracle(p)
    m = p.nvec
    x = xt - 0.25
    with G.Gadi.from_problem(p) as H:
        for op, which in [(G.OP_A, O.OP_A), (G.OP_M, O.OP_M), (G.OP_N, O.OP_N)]:
            y = torch.zeros(m, dtype=torch.float64, device="cuda")
            H.apply(op, dev64(x), y)
            assert np.array_equal(y.cpu().numpy(), orc.apply(which, x)), op
        # A^T of the real form: compare with the dense transpose
        y = torch.zeros(m, dtype=torch.float64, device="cuda")
        H.apply(G.OP_AT, dev64(x), y)
        if m <= 400:
            want = orc.dense(O.OP_A).T @ x
        else:
            want = orc.apply(O.OP_M, x) - orc.apply(O.OP_N, x)
        assert np.allclose(y.cpu().numpy(), want, rtol=1e-14, atol=1e-13)
        # host pointers give the same result as device pointers
        yh = np.zeros(m)
        H.apply(G.OP_A, x, yh)
        assert np.array_equal(yh, orc.apply(O.OP_A, x))


def _solve_h_pair(p, prec, alpha, rs, tol, maxit, stag):
    orc = O.Oracle(p)
    with G.Gadi.from_problem(p) as H:
        z = us_empty(p.nvec, prec)
        its = H.step_solve_h(alpha, prec, us_to_device(rs, prec), z, tol, maxit, stag)
        zg = us_to_host(z, prec)
    zo, it_o = orc.solve_h(alpha, prec, rs, tol, maxit, stag)
    return zg, its, zo, it_o


FIXED_TOL = {FP64: 1e-12, FP32: 2e-5, BF16: 0.06}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", PRECS)
def test_solve_h_fixed_iterations(case, prec):
    p, xt = CASES[case]()
    rs = rnd(prec, xt - 0.5)
    for its in (1, 4):
        zg, it_g, zo, it_o = _solve_h_pair(p, prec, 0.3, rs, 0.0, its, 0)
        # with tolerance 0 the oracle stops early only on an exactly zero
        # residual (a 1 x 1 grid after one step); the GPU's fused
        # multiply-add leaves the rounding error of that step instead, and
        # it may go on iterating on it up to the cap
        assert it_g == it_o or (it_o < its and it_o < it_g <= its), (it_g, it_o)
        err = np.linalg.norm(zg - zo) / np.linalg.norm(zo)
        assert err <= FIXED_TOL[prec] * its, (its, err)
        if its == 1 and prec == BF16:
            # one step: z = fl(a r); a differs only by the dot order
            assert np.all(np.abs(zg - zo) <= 1.01 * ulp_bf16(zo))


@pytest.mark.parametrize("case", ["2d_vec", "2d_wide", "2d_tall", "3d_vec", "cplx_vec", "csr"])
@pytest.mark.parametrize("prec", PRECS)
def test_solve_h_converged(case, prec):
    p, xt = CASES[case]()
    rs = rnd(prec, xt - 0.5)
    tol = 1e-2 if prec == BF16 else 1e-4
    zg, it_g, zo, it_o = _solve_h_pair(p, prec, 0.05, rs, tol, 1000, 10)
    assert abs(it_g - it_o) <= max(2, 0.2 * it_o), (it_g, it_o)
    orc = O.Oracle(p)

    def true_res(z):
        return np.linalg.norm(rs - (0.05 * z + orc.apply(O.OP_M, z))) / np.linalg.norm(rs)

    rg, ro = true_res(zg), true_res(zo)
    assert rg <= max(3 * ro, 3 * tol), (rg, ro)


def _solve_s_pair(p, prec, alpha, omega, z, tol, maxit, stag, pointwise):
    orc = O.Oracle(p)
    with G.Gadi.from_problem(p) as H:
        y = us_empty(p.nvec, prec)
        its = H.step_solve_s(alpha, omega, prec, us_to_device(z, prec), y, tol, maxit, stag, pointwise)
        yg = us_to_host(y, prec)
    yo, it_o = orc.solve_s(alpha, omega, prec, z, tol, maxit, stag, pointwise)
    return yg, its, yo, it_o


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", PRECS)
def test_solve_s_fixed_iterations(case, prec):
    p, xt = CASES[case]()
    z = rnd(prec, xt - 0.5)
    for its in (1, 4):
        yg, it_g, yo, it_o = _solve_s_pair(p, prec, 0.02, 0.7, z, 0.0, its, 0, False)
        # (an exactly zero residual stops the oracle early, as for H)
        assert it_g == it_o or (it_o < its and it_o < it_g <= its), (it_g, it_o)
        if np.linalg.norm(yo) == 0:
            assert np.linalg.norm(yg) == 0
            continue
        err = np.linalg.norm(yg - yo) / np.linalg.norm(yo)
        assert err <= FIXED_TOL[prec] * its, (its, err)


@pytest.mark.parametrize("case", ["cplx_vec", "cplx_odd", "cplx_pt"])
@pytest.mark.parametrize("prec", PRECS)
def test_solve_s_pointwise_bit_exact(case, prec):
    p, xt = CASES[case]()
    z = rnd(prec, xt - 0.5)
    yg, it_g, yo, it_o = _solve_s_pair(p, prec, 0.8, 1.0, z, 1e-3, 100, 10, True)
    assert it_g == it_o == 1
    assert np.array_equal(yg, yo)


@pytest.mark.parametrize("case", ["2d_vec", "2d_ragged", "3d_vec", "csr"])
@pytest.mark.parametrize("prec", PRECS)
def test_solve_s_converged(case, prec):
    p, xt = CASES[case]()
    z = rnd(prec, xt - 0.5)
    tol = 1e-2 if prec == BF16 else 1e-4
    alpha, omega = 0.02, 1.0
    yg, it_g, yo, it_o = _solve_s_pair(p, prec, alpha, omega, z, tol, 1000, 10, False)
    # Iteration counts are comparable only where the tolerance is attainable in
    # u_s (kappa(S^T S) u_s well below tol); beyond it both sides stop on the
    # stagnation rule at a rounding-dependent step and only the result matters.
    attainable = True
    if p.kind != 3:
        _, ks = G.condition_numbers(p, alpha)
        u = {FP64: 1.11e-16, FP32: 5.96e-8, BF16: 3.91e-3}[prec]
        attainable = ks * ks * u <= tol / 10
    if attainable:
        assert abs(it_g - it_o) <= max(2, 0.2 * it_o), (it_g, it_o)
    orc = O.Oracle(p)
    gvec = (2 - omega) * alpha * z

    def true_res(y):
        return np.linalg.norm(gvec - (alpha * y + orc.apply(O.OP_N, y))) / np.linalg.norm(gvec)

    rg, ro = true_res(yg), true_res(yo)
    assert rg <= max(3 * ro, 30 * tol), (rg, ro)


def test_integer_pipe_conversions_match_hardware():
    """The binary32/BF16 <-> binary64 conversions the FP64 residual uses are
    assembled from IEEE 754 fields on the integer pipe; they must equal the
    hardware conversions bit for bit: random bit patterns over every exponent,
    round-to-nearest-even ties at the binary32 and BF16 cut, the ends of the
    binary32 range (smallest normal, largest finite, the tie that rounds to
    infinity), zeros, subnormals, infinities and NaNs."""
    import torch
    g = np.random.default_rng(77)
    pats = [g.integers(0, 2**63, 200000, dtype=np.uint64) * np.uint64(2) + g.integers(0, 2, 200000, dtype=np.uint64)]
    # exponents near the binary32 range ends, random significands
    for e in list(range(890, 905)) + list(range(1140, 1155)):
        m = g.integers(0, 2**52, 2000, dtype=np.uint64)
        for sgn in (0, 1):
            pats.append((np.uint64(sgn) << np.uint64(63)) | (np.uint64(e) << np.uint64(52)) | m)
    # exact ties and neighbours at the binary32 (bit 29) and BF16 (bit 45) cuts
    base = g.integers(0, 2**52, 4000, dtype=np.uint64)
    exps = g.integers(880, 1170, 4000, dtype=np.uint64) << np.uint64(52)
    for cut in (29, 45):
        hm = ~np.uint64((1 << cut) - 1) & np.uint64((1 << 52) - 1)
        tie = (base & hm) | np.uint64(1 << (cut - 1))
        for t in (tie, tie - np.uint64(1), tie + np.uint64(1)):
            pats.append(exps | t)
    specials = np.array([0.0, -0.0, 2.0 ** -126, -(2.0 ** -126), 2.0 ** -127, 2.0 ** -149, 2.0 ** -150,
                         np.nextafter(2.0 ** -126, 0), (2 - 2.0 ** -23) * 2.0 ** 127,
                         (2 - 2.0 ** -24) * 2.0 ** 127, np.nextafter((2 - 2.0 ** -24) * 2.0 ** 127, 0),
                         (2 - 2.0 ** -8) * 2.0 ** 127, np.nextafter((2 - 2.0 ** -8) * 2.0 ** 127, 0),
                         2.0 ** 128, np.inf, -np.inf, np.nan, 5e-324, 1e-310, 1.0, -1.5, 3.0e38])
    pats.append(specials.view(np.uint64))
    allp = np.concatenate(pats).view(np.float64)
    d = torch.from_numpy(allp.copy()).cuda()
    assert G.selftest_convert(d) == [0, 0, 0, 0]
    # float bit patterns across the whole range (every exponent, both signs,
    # subnormals, infinities) in their low 32 bits: the BF16 rounding by
    # instruction equals the integer sequence
    pats32 = np.arange(0, 2 ** 32, 4099, dtype=np.uint64)
    assert G.selftest_convert(torch.from_numpy(pats32.view(np.float64)).cuda())[3] == 0


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", PRECS)
def test_residual_double_fp64_bit_exact(case, prec):
    """The residual in double-FP64 (u_r ~ u^2): x_out, both parts of r, r_s and
    ||r|| against the oracle, element by element, with b close to A x so the
    residual cancels and its low part matters."""
    import torch
    p, xt = CASES[case]()
    orc = O.Oracle(p)
    m = p.nvec
    g = SplitMix64(17)
    x = g.uniform_array(m) - 0.5
    y = rnd(prec, (g.uniform_array(m) - 0.5) * 1e-2)
    b = orc.rhs(x + y) + (g.uniform_array(m) - 0.5) * 1e-10
    with G.Gadi.from_problem(p) as H:
        xo = torch.zeros(m, dtype=torch.float64, device="cuda")
        rh, rl = torch.zeros_like(xo), torch.zeros_like(xo)
        rs = us_empty(m, prec)
        nrm = H.step_residual_ur(G.FP64X2, prec, dev64(b), dev64(x), us_to_device(y, prec), xo, rh, rl, rs)
        # u_r = FP64 through the same entry point: the low part is zero
        rl2 = torch.ones_like(xo)
        H.step_residual_ur(G.FP64, prec, dev64(b), dev64(x), us_to_device(y, prec), xo, rh.clone(), rl2,
                           us_empty(m, prec))
        assert not torch.any(rl2 != 0)
    xo_o, rh_o, rl_o, rs_o, n_o = orc.residual_dd(prec, b, x, y)
    assert np.array_equal(xo.cpu().numpy(), xo_o)
    assert np.array_equal(rh.cpu().numpy(), rh_o)
    assert np.array_equal(rl.cpu().numpy(), rl_o)
    assert np.array_equal(us_to_host(rs, prec), rs_o)
    assert abs(nrm - n_o) <= 1e-12 * n_o
