"""Element-by-element GPU parity of one inner step (CG on H, CGNR on S)
against the oracle.

Two kinds of input:

* exact inputs: small dyadic right-hand sides (and dyadic coefficients), with
  enough zeros that every product and every partial sum of the step is exact
  in the compute type.  The only roundings left are those of the same exact
  values on both sides (the scalar a = rr / pq, the stored vectors), so one
  step must give the same bits, in every precision, on every operator class
  and kernel form (streaming, SM-resident, tensor-memory resident, narrow
  rows, two column passes, 3D, complex, CSR).

* random inputs: the GPU sums its dot products in a tree and fuses
  multiply-adds, the oracle takes the float nearest to the exact dot (FP32)
  or sums sequentially (FP64).  Each element must then agree within 2 ulp of
  u_s plus the bound the dot products allow on the step's scalar: for a dot
  s = sum t_i, |s_gpu - s_orc| <= (gamma_gpu + gamma_orc) sum |t_i|, with the
  GPU's tree of depth L = ceil(log2 m) + 1 and the oracle's error (u/2 for
  FP32, m u for FP64), plus 3 u per element where the GPU's fused H p or
  S^T u differs from the oracle's separately rounded one.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_2512_21164_gb300 as G
from helpers import BF16, FP32, FP64, PRECS, us_empty, us_to_device, us_to_host
from workloads import K_2D5, K_3D7, K_C2D5, K_CSR, Problem, SplitMix64, conv_diff_2d, conv_diff_3d

pytestmark = pytest.mark.gpu

U = {FP64: 2.0 ** -53, FP32: 2.0 ** -24, BF16: 2.0 ** -24}  # compute-type unit roundoff


def _dyadic_csr(n, seed):
    """A sparse nonsymmetric matrix with dyadic entries (multiples of 1/8)
    and a diagonally dominant symmetric part."""
    g = SplitMix64(seed)
    rows = []
    for i in range(n):
        r = {}
        for _ in range(3):
            j = int(g.uniform() * n)
            if j != i:
                r[j] = (int(g.uniform() * 9) - 4) / 8.0
        rows.append(r)
    rp, cl, vl = [0], [], []
    for i, r in enumerate(rows):
        r = dict(r)
        r[i] = 4.0
        for j in sorted(r):
            cl.append(j)
            vl.append(r[j])
        rp.append(len(cl))
    return Problem(K_CSR, n, rowptr=np.asarray(rp, np.int32), col=np.asarray(cl, np.int32),
                   val=np.asarray(vl, np.float64))


# grids chosen for the kernel forms they take with one block per SM: the
# tall ones have more rows than SMs (the resident H-solve), 2560 x 200 two
# column passes, 8 x 400 rows narrower than a block
H_CASES = {
    "2d_vec": lambda: Problem(K_2D5, 64, 48, 1, 1.0 / 65, (30.0, 50.0, 0.0)),
    "2d_ragged": lambda: Problem(K_2D5, 37, 5, 1, 1.0 / 38, (30.0, 50.0, 0.0)),
    "2d_tall": lambda: Problem(K_2D5, 64, 700, 1, 1.0 / 65, (30.0, 50.0, 0.0)),
    "2d_wide_tall": lambda: Problem(K_2D5, 2560, 200, 1, 1.0 / 2561, (30.0, 50.0, 0.0)),
    "2d_narrow_tall": lambda: Problem(K_2D5, 8, 400, 1, 1.0 / 9, (30.0, 50.0, 0.0)),
    "3d_vec": lambda: Problem(K_3D7, 16, 16, 16, 1.0 / 17, (10.0, 10.0, 10.0)),
    "3d_ragged": lambda: Problem(K_3D7, 7, 5, 9, 1.0 / 8, (13.0, 29.0, 41.0)),
    # 16-byte rows in every precision (FP32: the plane-ring sweep) with a
    # partial last y-tile (40 = 16 + 16 + 8 rows) and a partial strip, z runs
    # that cross from one column to the next; and rows of two strips
    "3d_tiles": lambda: Problem(K_3D7, 24, 40, 200, 1.0 / 25, (10.0, 20.0, 30.0)),
    "3d_strips": lambda: Problem(K_3D7, 136, 17, 30, 1.0 / 137, (10.0, 20.0, 30.0)),
    "cplx_vec": lambda: Problem(K_C2D5, 32, 32, 1, 1.0 / 33, (0.0, 0.0, 0.0), 2.0, 40.0),
    "csr": lambda: _dyadic_csr(500, 9),
}
# S-solve cases with c_i = beta_i h / 2 = 1/2 (h = 1/8, beta = 8): S = (I + N') / 2
S_CASES = {
    "2d_vec": lambda: Problem(K_2D5, 64, 48, 1, 0.125, (8.0, 8.0, 0.0)),
    "2d_ragged": lambda: Problem(K_2D5, 37, 5, 1, 0.125, (8.0, 8.0, 0.0)),
    "2d_tall": lambda: Problem(K_2D5, 64, 700, 1, 0.125, (8.0, 8.0, 0.0)),
    "3d_vec": lambda: Problem(K_3D7, 16, 16, 16, 0.125, (8.0, 8.0, 8.0)),
    "3d_tiles": lambda: Problem(K_3D7, 24, 40, 200, 0.125, (8.0, 8.0, 8.0)),
    "3d_strips": lambda: Problem(K_3D7, 136, 17, 30, 0.125, (8.0, 8.0, 8.0)),
    "csr": lambda: _dyadic_csr(500, 11),
}


def _sparse_dyadic(m, nonzero, kmax, seed):
    """k/8 with k uniform in [-kmax, kmax] \\ {0} at `nonzero` random positions."""
    g = SplitMix64(seed)
    v = np.zeros(m)
    for _ in range(nonzero):
        k = 0
        while k == 0:
            k = int(g.uniform() * (2 * kmax + 1)) - kmax
        v[int(g.uniform() * m)] = k / 8.0
    return v


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2512_21164_gb300 import build
    build.build()


def _h_step(p, prec, alpha, rs):
    orc = O.Oracle(p)
    with G.Gadi.from_problem(p) as H:
        z = us_empty(p.nvec, prec)
        its = H.step_solve_h(alpha, prec, us_to_device(rs, prec), z, 0.0, 1, 0)
        zg = us_to_host(z, prec)
    zo, it_o = orc.solve_h(alpha, prec, rs, 0.0, 1, 0)
    assert its == it_o == 1
    return zg, zo


def _s_step(p, prec, alpha, omega, z):
    orc = O.Oracle(p)
    with G.Gadi.from_problem(p) as H:
        y = us_empty(p.nvec, prec)
        its = H.step_solve_s(alpha, omega, prec, us_to_device(z, prec), y, 0.0, 1, 0, False)
        yg = us_to_host(y, prec)
    yo, it_o = orc.solve_s(alpha, omega, prec, z, 0.0, 1, 0, False)
    assert its == it_o == 1
    return yg, yo


@pytest.mark.parametrize("case", list(H_CASES))
@pytest.mark.parametrize("prec", PRECS)
def test_solve_h_one_step_same_bits_on_exact_inputs(case, prec):
    """rs = k/8 (|k| <= 7) at <= 4000 points, alpha = 1/4: H p and both dot
    products are exact in FP32 (partial sums stay below 2^15 in units of
    2^-8), so z = fl(a p) must agree bit for bit."""
    p = H_CASES[case]()
    rs = _sparse_dyadic(p.nvec, min(p.nvec, 4000), 7, 501)
    zg, zo = _h_step(p, prec, 0.25, rs)
    assert np.array_equal(zg, zo), np.max(np.abs(zg - zo))


@pytest.mark.parametrize("case", list(S_CASES))
@pytest.mark.parametrize("prec", PRECS)
def test_solve_s_one_step_same_bits_on_exact_inputs(case, prec):
    """z = +-1/8 at <= 800 points, alpha = 1/2, omega = 1, c_i = 1/2 (CSR:
    eighths): g, S^T g, S p and the two dot products are exact in FP32, so
    y = fl(a p) must agree bit for bit."""
    p = S_CASES[case]()
    z = _sparse_dyadic(p.nvec, min(p.nvec // 4, 800), 1, 502)
    yg, yo = _s_step(p, prec, 0.5, 1.0, z)
    assert np.array_equal(yg, yo), np.max(np.abs(yg - yo))


def _ulp(prec, a):
    e = np.floor(np.log2(np.maximum(np.abs(a), 2.0 ** -126)))
    return 2.0 ** (e - {FP64: 52, FP32: 23, BF16: 7}[prec])


def _dot_bound(prec, m, kappa):
    """Relative bound on the difference of the GPU's and the oracle's value of
    a dot product whose terms have sum |t_i| = kappa |sum t_i|."""
    u = U[prec]
    L = math.ceil(math.log2(max(m, 2))) + 1
    orc = 0.5 * u if prec != FP64 else m * u
    return (L * u + orc) * kappa


RAND_CASES = {
    "2d_vec": lambda: conv_diff_2d(64, 101, ny=48),
    "2d_tall": lambda: conv_diff_2d(64, 112, ny=700),
    "2d_wide_tall": lambda: conv_diff_2d(2560, 117, ny=200),
    "3d_vec": lambda: conv_diff_3d(16, 106),
    "3d_tiles": lambda: (Problem(K_3D7, 24, 40, 200, 1.0 / 25, (10.0, 20.0, 30.0)),
                         SplitMix64(118).uniform_array(24 * 40 * 200)),
}


@pytest.mark.parametrize("case", list(RAND_CASES))
@pytest.mark.parametrize("prec", [FP64, FP32])
def test_solve_h_one_step_elementwise_random(case, prec):
    p, xt = RAND_CASES[case]()
    rs = np.asarray(xt - 0.5, np.float64)
    if prec == FP32:
        rs = rs.astype(np.float32).astype(np.float64)
    alpha = 0.3
    zg, zo = _h_step(p, prec, alpha, rs)
    orc = O.Oracle(p)
    q = alpha * rs + orc.apply(O.OP_M, rs)
    m = p.nvec
    kap_pq = np.sum(np.abs(rs * q)) / abs(np.dot(rs, q))
    # a = rr / pq: both dots, plus the fused H p (3 u per element)
    d = _dot_bound(prec, m, 1.0) + _dot_bound(prec, m, kap_pq) + 3 * U[prec] * kap_pq + 2 * U[prec]
    tol = 2 * _ulp(prec, zo) + d * np.abs(zo)
    bad = np.abs(zg - zo) > tol
    assert not np.any(bad), (np.sum(bad), np.max(np.abs(zg - zo) / _ulp(prec, zo)))


def _abs_n(p, v):
    """|N| |v| for the real stencil classes: sum over neighbours of
    |c_i| |v_nbr| with c_i = beta_i h / 2 (zero outside the grid)."""
    dims = (p.nz, p.ny, p.nx) if p.kind == K_3D7 else (p.ny, p.nx)
    a = np.abs(v).reshape(dims)
    out = np.zeros_like(a)
    axes = list(range(len(dims)))[::-1]  # x, y (, z)
    for k, ax in enumerate(axes):
        c = abs(p.beta[k] * p.hh / 2.0)
        lo = [slice(None)] * len(dims)
        hi = [slice(None)] * len(dims)
        lo[ax], hi[ax] = slice(0, -1), slice(1, None)
        out[tuple(lo)] += c * a[tuple(hi)]
        out[tuple(hi)] += c * a[tuple(lo)]
    return out.ravel()


@pytest.mark.parametrize("case", ["2d_vec", "2d_tall", "3d_vec", "3d_tiles"])
@pytest.mark.parametrize("prec", [FP64, FP32])
def test_solve_s_one_step_elementwise_random(case, prec):
    p, xt = RAND_CASES[case]()
    z = np.asarray(xt - 0.5, np.float64)
    if prec == FP32:
        z = z.astype(np.float32).astype(np.float64)
    alpha, omega = 0.02, 0.7
    yg, yo = _s_step(p, prec, alpha, omega, z)
    m = p.nvec
    orc = O.Oracle(p)
    g = (2 - omega) * alpha * z
    t0 = alpha * g - orc.apply(O.OP_N, g)
    uvec = alpha * t0 + orc.apply(O.OP_N, t0)
    a = np.dot(t0, t0) / np.dot(uvec, uvec)
    # t_0 = fl(S^T g) may differ by a few roundings of the row's terms (fused
    # on the GPU), which cancel where t_0 is small: |dt_0| <= 4 u (alpha |g| +
    # |N| |g|), carried into y = a t_0; the scalar a = tt / uu differs by the
    # bound of two sums of squares; both sides round y once more
    cond = alpha * np.abs(g) + _abs_n(p, g)
    d = 2 * _dot_bound(prec, m, 1.0) + 8 * U[prec]
    tol = 4 * _ulp(prec, yo) + d * np.abs(yo) + 4 * U[prec] * abs(a) * cond
    bad = np.abs(yg - yo) > tol
    assert not np.any(bad), (np.sum(bad), np.max(np.abs(yg - yo) / _ulp(prec, yo)))
