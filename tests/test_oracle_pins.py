"""Pins of the CPU oracle against facts fixed by the paper or by mathematics.

Each test checks the oracle against something other than itself: printed
values (Table 1), closed forms (Sec. 2.1 iteration matrix, HSS bounds),
dense direct solves, textbook Kronecker constructions of the discretisations
(Sec. 5.2-5.4), brute force over every BF16 value, and invariants (M + N = A,
M = M^T, N = -N^T, Lemma 1).  A dropped term, wrong sign, wrong index or
transposed operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from workloads import (K_2D5, K_3D7, K_C2D5, K_CSR, Problem, SplitMix64, alpha_star,
                       complex_rd, conv_diff_2d, conv_diff_3d, random_csr)

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# rounding emulation
# --------------------------------------------------------------------------
def _all_bf16_values():
    bits = np.arange(0, 1 << 16, dtype=np.uint32) << np.uint32(16)
    v = bits.view(np.float32).astype(np.float64)
    return v


def _bf16_brute(x, table):
    """Nearest finite BF16 to x, ties to the value with an even last bit
    (searched over all 65536 encodings)."""
    fin = table[np.isfinite(table)]
    enc = np.arange(1 << 16)[np.isfinite(table)]
    d = np.abs(fin - x)
    best = d.min()
    cand = np.where(d == best)[0]
    if len(cand) > 1:
        even = [c for c in cand if enc[c] % 2 == 0]
        cand = even if even else cand
    return fin[cand[0]]


def test_bf16_special_cases():
    r = O.round_bf16
    assert r(1.0 + 2.0 ** -8) == 1.0                       # tie -> even
    assert r(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6       # tie -> even (up)
    assert r(1.0 + 3 * 2.0 ** -9) == 1.0 + 2.0 ** -7       # above half -> up
    assert r(1.0 + 2.0 ** -8 + 2.0 ** -30) == 1.0 + 2.0 ** -7
    maxbf = (2 - 2.0 ** -7) * 2.0 ** 127
    assert r(maxbf) == maxbf
    assert r(-maxbf) == -maxbf
    assert math.isinf(r(maxbf * (1 + 2.0 ** -8)))          # halfway above max -> inf
    assert r(maxbf * (1 + 2.0 ** -9)) == maxbf
    assert math.isnan(r(float("nan")))
    assert r(float("inf")) == float("inf")
    assert r(0.0) == 0.0
    assert r(2.0 ** -133) == 2.0 ** -133                   # smallest subnormal
    assert r(2.0 ** -134) == 0.0                           # tie -> even (zero)
    assert r(1.5 * 2.0 ** -134) == 2.0 ** -133


def test_bf16_brute_force():
    table = _all_bf16_values()
    g = SplitMix64(11)
    xs = []
    for _ in range(300):
        e = int(g.uniform() * 60) - 30
        xs.append((2 * g.uniform() - 1) * 2.0 ** e)
    # exact ties and near-ties
    for k in range(40):
        base = table[0x3F80 + k]
        nxt = table[0x3F80 + k + 1]
        xs += [(base + nxt) / 2, (base + nxt) / 2 * (1 + 1e-12), -(base + nxt) / 2]
    xs += [2.0 ** -130 * 1.37, -(2.0 ** -128) * 0.51]
    for x in xs:
        assert O.round_bf16(x) == _bf16_brute(x, table), x


def test_fp32_rounding_matches_numpy():
    g = SplitMix64(12)
    for _ in range(500):
        x = (2 * g.uniform() - 1) * 2.0 ** (int(g.uniform() * 200) - 100)
        assert O.round_prec(O.FP32, x) == float(np.float32(x))


def test_unit_roundoff_table1():
    """Largest relative error of the emulated roundings vs Table 1's u."""
    rows = [l.split() for l in open(os.path.join(GOLD, "table1_unit_roundoff.txt"))
            if l.strip() and not l.startswith("#")]
    u = {name: float(val) for name, _, val in rows}
    g = SplitMix64(13)
    xs = np.array([1.0 + g.uniform() for _ in range(20000)])
    err_bf = max(abs(O.round_bf16(x) - x) / abs(x) for x in xs)
    err_32 = max(abs(O.round_prec(O.FP32, x) - x) / abs(x) for x in xs)
    assert err_bf <= u["bf16"] * (1 + 1e-3) and err_bf > 0.9 * u["bf16"]
    assert err_32 <= u["fp32"] * (1 + 1e-3) and err_32 > 0.9 * u["fp32"]
    assert abs(u["fp64"] - 2.0 ** -53) / 2.0 ** -53 < 0.01


# --------------------------------------------------------------------------
# operators: stencil == textbook Kronecker construction
# --------------------------------------------------------------------------
def _tri(n, sub, diag, sup):
    return (np.diag(np.full(n, diag)) + np.diag(np.full(n - 1, sub), -1)
            + np.diag(np.full(n - 1, sup), 1))


def _kron_2d(p):
    """A = I (x) T_x + T_y (x) I for x-fastest ordering (Sec. 5.2's Kronecker
    form) with T_i = Tridiag(-1 - c_i, 2, -1 + c_i), c_i = beta_i h / 2."""
    h = p.hh
    cx, cy = p.beta[0] * h / 2, p.beta[1] * h / 2
    Tx = _tri(p.nx, -1 - cx, 2.0, -1 + cx)
    Ty = _tri(p.ny, -1 - cy, 2.0, -1 + cy)
    return np.kron(np.eye(p.ny), Tx) + np.kron(Ty, np.eye(p.nx))


def _kron_3d(p):
    h = p.hh
    c = [b * h / 2 for b in p.beta]
    T = [_tri(n, -1 - ci, 2.0, -1 + ci) for n, ci in zip((p.nx, p.ny, p.nz), c)]
    Ix, Iy, Iz = np.eye(p.nx), np.eye(p.ny), np.eye(p.nz)
    return (np.kron(Iz, np.kron(Iy, T[0])) + np.kron(Iz, np.kron(T[1], Ix))
            + np.kron(T[2], np.kron(Iy, Ix)))


@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 3), (7, 5), (9, 9)])
def test_stencil_2d_equals_kronecker(nx, ny):
    p, _ = conv_diff_2d(nx, 21, beta=(37.0, -13.0), ny=ny)
    orc = O.Oracle(p)
    A = orc.dense(O.OP_A)
    K = _kron_2d(p)
    assert np.allclose(A, K, rtol=0, atol=1e-15)
    M, N = orc.dense(O.OP_M), orc.dense(O.OP_N)
    assert np.array_equal(M + N, A)           # M + N = A (coefficients built so)
    assert np.array_equal(M, M.T)             # HSS: symmetric part
    assert np.array_equal(N, -N.T)            # HSS: skew part
    assert np.allclose(M, (K + K.T) / 2, atol=1e-15)
    assert np.allclose(N, (K - K.T) / 2, atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 4])
def test_stencil_3d_equals_kronecker(n):
    p = Problem(K_3D7, n, n + 1, n + 2, 1.0 / (n + 1), (3.0, 11.0, -7.0))
    orc = O.Oracle(p)
    A = orc.dense(O.OP_A)
    K = _kron_3d(p)
    assert np.allclose(A, K, rtol=0, atol=1e-15)
    M, N = orc.dense(O.OP_M), orc.dense(O.OP_N)
    assert np.array_equal(M + N, A)
    assert np.array_equal(M, M.T) and np.array_equal(N, -N.T)


def test_complex_operator_equals_complex_matrix():
    p, _ = complex_rd(5, 31, kappa=2.5, sigma=7.0)
    orc = O.Oracle(p)
    n = p.npoints
    L = np.kron(np.eye(5), _tri(5, -1, 2, -1)) + np.kron(_tri(5, -1, 2, -1), np.eye(5))
    Wc = L + 2.5 * np.eye(n) + 1j * 7.0 * np.eye(n)
    g = SplitMix64(5)
    x = g.uniform_array(2 * n) - 0.5
    xc = x[0::2] + 1j * x[1::2]
    y = orc.apply(O.OP_A, x)
    yc = Wc @ xc
    assert np.allclose(y[0::2], yc.real, atol=1e-13) and np.allclose(y[1::2], yc.imag, atol=1e-13)
    # real block form (Sec. 5.4) restricted to interleaving: M symmetric, N skew
    M, N = orc.dense(O.OP_M), orc.dense(O.OP_N)
    assert np.array_equal(M, M.T) and np.array_equal(N, -N.T)
    assert np.array_equal(M + N, orc.dense(O.OP_A))


def test_csr_apply_and_split():
    import scipy.sparse as sp
    p, xt = random_csr(60, 41)
    orc = O.Oracle(p)
    A = sp.csr_matrix((p.val, p.col, p.rowptr), shape=(60, 60))
    assert np.allclose(orc.apply(O.OP_A, xt), A @ xt, rtol=1e-15, atol=1e-13)
    Md, Nd, Ad = orc.dense(O.OP_M), orc.dense(O.OP_N), A.toarray()
    assert np.array_equal(Md, Md.T) and np.array_equal(Nd, -Nd.T)
    assert np.max(np.abs(Md + Nd - Ad)) <= 2.0 ** -52 * np.max(np.abs(Ad))
    assert np.min(np.linalg.eigvalsh(Md)) > 0         # positive definite symmetric part


# --------------------------------------------------------------------------
# inner solvers vs dense direct solves
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["2d", "3d", "cplx", "csr"])
def test_inner_solves_equal_dense(kind):
    if kind == "2d":
        p, xt = conv_diff_2d(9, 51, ny=7)
    elif kind == "3d":
        p, xt = conv_diff_3d(4, 52)
    elif kind == "cplx":
        p, xt = complex_rd(6, 53)
    else:
        p, xt = random_csr(50, 54)
    orc = O.Oracle(p)
    M, N = orc.dense(O.OP_M), orc.dense(O.OP_N)
    I = np.eye(M.shape[0])
    alpha, omega = 0.37, 0.6
    r = xt - 0.5
    z, its = orc.solve_h(alpha, O.FP64, r, tol=1e-14, maxit=2000, stag=0)
    assert its <= 2 * M.shape[0] + 5
    zd = np.linalg.solve(alpha * I + M, r)
    assert np.linalg.norm(z - zd) <= 1e-11 * np.linalg.norm(zd)
    y, its = orc.solve_s(alpha, omega, O.FP64, z, tol=1e-14, maxit=2000, stag=0)
    yd = np.linalg.solve(alpha * I + N, (2 - omega) * alpha * zd)
    assert np.linalg.norm(y - yd) <= 1e-10 * np.linalg.norm(yd)


def test_pointwise_s_solve_equals_cgnr_complex():
    p, xt = complex_rd(6, 55)
    orc = O.Oracle(p)
    z = xt - 0.5
    y1, it1 = orc.solve_s(0.8, 1.0, O.FP64, z, tol=1e-14, maxit=100, stag=0, pointwise=True)
    y2, it2 = orc.solve_s(0.8, 1.0, O.FP64, z, tol=1e-14, maxit=100, stag=0)
    assert it1 == 1 and it2 <= 2  # S = (alpha + i sigma) I: CGNR ends in one step
    assert np.allclose(y1, y2, rtol=1e-13, atol=1e-15)
    # closed form y = (2 - omega) alpha z / (alpha + i sigma)
    zc = z[0::2] + 1j * z[1::2]
    yc = 0.8 * zc / (0.8 + 1j * p.sigma)
    assert np.allclose(y1[0::2], yc.real, atol=1e-14) and np.allclose(y1[1::2], yc.imag, atol=1e-14)


def test_beta_zero_cgnr_one_step():
    """N = 0: S = alpha I, CGNR converges in one step and y = (2 - omega) z."""
    p, xt = conv_diff_2d(8, 56, beta=(0.0, 0.0))
    orc = O.Oracle(p)
    y, its = orc.solve_s(0.3, 0.5, O.FP64, xt, tol=1e-14, maxit=10, stag=0)
    assert its == 1
    assert np.allclose(y, 1.5 * xt, rtol=1e-14)


def test_low_precision_storage_is_representable():
    p, xt = conv_diff_2d(12, 57)
    orc = O.Oracle(p)
    rs = np.array([O.round_bf16(v) for v in xt])
    z, _ = orc.solve_h(0.2, O.BF16, rs, tol=1e-2)
    assert all(O.round_bf16(v) == v for v in z)
    y, _ = orc.solve_s(0.2, 1.0, O.BF16, z, tol=1e-2)
    assert all(O.round_bf16(v) == v for v in y)
    z32, _ = orc.solve_h(0.2, O.FP32, xt.astype(np.float32).astype(np.float64), tol=1e-3)
    assert np.array_equal(z32.astype(np.float32).astype(np.float64), z32)


def test_low_precision_inner_solve_accuracy():
    """FP32 / BF16 inner CG reaches its tolerance in terms of the true residual
    up to the storage rounding (c kappa(H) u_s)."""
    p, xt = conv_diff_2d(16, 58)
    orc = O.Oracle(p)
    M = orc.dense(O.OP_M)
    H = 0.5 * np.eye(M.shape[0]) + M
    r = np.array([O.round_prec(O.FP32, v) for v in xt])
    for prec, tol, slack in [(O.FP32, 1e-4, 1e-3), (O.BF16, 1e-2, 0.1)]:
        rs = np.array([O.round_prec(prec, v) for v in r])
        z, _ = orc.solve_h(0.5, prec, rs, tol=tol)
        res = np.linalg.norm(rs - H @ z) / np.linalg.norm(rs)
        assert res <= slack, (prec, res)


# --------------------------------------------------------------------------
# Algorithm 1 vs the GADI definition
# --------------------------------------------------------------------------
def _tiny(kind):
    if kind == "2d":
        return conv_diff_2d(8, 61, ny=6)
    if kind == "3d":
        return conv_diff_3d(4, 62)
    if kind == "cplx":
        return complex_rd(5, 63)
    return random_csr(40, 64)


@pytest.mark.parametrize("kind", ["2d", "3d", "cplx", "csr"])
def test_alg1_equals_two_step_form(kind):
    p, xt = _tiny(kind)
    orc = O.Oracle(p)
    A, M, N = orc.dense(O.OP_A), orc.dense(O.OP_M), orc.dense(O.OP_N)
    b = orc.rhs(xt)
    assert np.allclose(b, A @ xt, rtol=1e-14, atol=1e-14)
    for alpha, omega in [(0.3, 0.0), (1.1, 1.0), (0.05, 1.7)]:
        xs1 = O.alg1_dense(A, M, N, b, alpha, omega, 6)
        xs2 = O.two_step_gadi(A, M, N, b, alpha, omega, 6)
        for a1, a2 in zip(xs1, xs2):
            assert np.linalg.norm(a1 - a2) <= 1e-12 * max(1.0, np.linalg.norm(a2))


@pytest.mark.parametrize("kind", ["2d", "3d", "cplx", "csr"])
def test_oracle_gadi_equals_dense_alg1(kind):
    """The oracle's Algorithm 1 with FP64 and tight inner solves reproduces
    the iterates of Algorithm 1 with dense direct subsolves."""
    p, xt = _tiny(kind)
    orc = O.Oracle(p)
    A, M, N = orc.dense(O.OP_A), orc.dense(O.OP_M), orc.dense(O.OP_N)
    b = orc.rhs(xt)
    alpha, omega = 0.4, 0.8
    xs = O.alg1_dense(A, M, N, b, alpha, omega, 5)
    for k in range(1, 6):
        x, st = orc.gadi(b, alpha, omega, O.FP64, tol=0.0, maxit=k, tol_h=1e-15, tol_s=1e-15,
                         maxit_inner=5000, inner_stag=0, outer_stag_window=0)
        assert st["outer_its"] == k and st["status"] == "NOT_CONVERGED"
        assert np.linalg.norm(x - xs[k]) <= 1e-10 * np.linalg.norm(xs[k])
        # relres history equals ||b - A x_j|| / ||b||
        for j in range(k + 1):
            rj = np.linalg.norm(b - A @ xs[j]) / np.linalg.norm(b)
            assert abs(st["history"][j] - rj) <= 1e-9 * rj + 1e-15


def test_fixed_point():
    """From x0 = A^-1 b one iteration moves x by at most c kappa(A) u."""
    p, xt = conv_diff_2d(10, 65)
    orc = O.Oracle(p)
    A = orc.dense(O.OP_A)
    b = orc.rhs(xt)
    xs = np.linalg.solve(A, b)
    kap = np.linalg.cond(A)
    x1, st = orc.gadi(b, 0.3, 1.0, O.FP64, tol=0.0, maxit=1, x0=xs, tol_h=1e-14, tol_s=1e-14,
                      inner_stag=0, outer_stag_window=0)
    assert np.linalg.norm(x1 - xs) <= 100 * kap * 2.0 ** -53 * np.linalg.norm(xs)


# --------------------------------------------------------------------------
# iteration matrix: Lemma 1, closed forms, Remark 1
# --------------------------------------------------------------------------
def test_lemma1_spectral_radius_below_one():
    p, _ = conv_diff_2d(7, 71, ny=6)
    orc = O.Oracle(p)
    A, M, N = orc.dense(O.OP_A), orc.dense(O.OP_M), orc.dense(O.OP_N)
    lam = np.linalg.eigvalsh(M)
    for alpha in [0.01, 0.1, 0.5, 1.0, 10.0]:
        T0 = O.iteration_matrix(A, M, N, alpha, 0.0)
        rho0 = max(abs(np.linalg.eigvals(T0)))
        # HSS bound rho(T_F(alpha,0)) <= max |alpha - lambda| / (alpha + lambda) over eig(M)
        assert rho0 <= max(abs(alpha - lam) / (alpha + lam)) + 1e-12
        for omega in [0.0, 0.5, 1.0, 1.5, 1.9]:
            T = O.iteration_matrix(A, M, N, alpha, omega)
            assert max(abs(np.linalg.eigvals(T))) < 1.0
            # T_F(alpha, omega) = (omega/2) I + (1 - omega/2) T_F(alpha, 0)
            assert np.allclose(T, omega / 2 * np.eye(len(A)) + (1 - omega / 2) * T0, atol=1e-12)


def test_beta_zero_closed_form_spectrum():
    """N = 0: eig(T_F) = (alpha - (1 - omega) lambda) / (alpha + lambda) with the
    Laplacian eigenvalues lambda_jk = 4 sin^2(j pi h/2) + 4 sin^2(k pi h/2)."""
    n = 6
    p, _ = conv_diff_2d(n, 72, beta=(0.0, 0.0))
    orc = O.Oracle(p)
    A, M, N = orc.dense(O.OP_A), orc.dense(O.OP_M), orc.dense(O.OP_N)
    h = 1.0 / (n + 1)
    lam = np.array([4 * math.sin(j * math.pi * h / 2) ** 2 + 4 * math.sin(k * math.pi * h / 2) ** 2
                    for j in range(1, n + 1) for k in range(1, n + 1)])
    for alpha, omega in [(0.5, 1.0), (2.0, 0.3)]:
        mu = np.sort((alpha - (1 - omega) * lam) / (alpha + lam))
        ev = np.sort(np.linalg.eigvals(O.iteration_matrix(A, M, N, alpha, omega)).real)
        assert np.allclose(ev, mu, atol=1e-12)
    assert math.isclose(alpha_star(p), math.sqrt(lam.min() * lam.max()), rel_tol=1e-12)


def test_complex_closed_form_spectrum():
    """W = L + kappa I, T = sigma I commute: mu_jk = 1 - (2 - omega) alpha (w + i sigma)
    / ((alpha + w)(alpha + i sigma)); the real block form has each mu and its conjugate."""
    n = 4
    p, _ = complex_rd(n, 73, kappa=1.5, sigma=20.0)
    orc = O.Oracle(p)
    A, M, N = orc.dense(O.OP_A), orc.dense(O.OP_M), orc.dense(O.OP_N)
    h = 1.0 / (n + 1)
    w = np.array([4 * math.sin(j * math.pi * h / 2) ** 2 + 4 * math.sin(k * math.pi * h / 2) ** 2
                  for j in range(1, n + 1) for k in range(1, n + 1)]) + 1.5
    alpha, omega = 3.0, 1.0
    mu = 1 - (2 - omega) * alpha * (w + 20j) / ((alpha + w) * (alpha + 20j))
    ev = np.linalg.eigvals(O.iteration_matrix(A, M, N, alpha, omega))
    want = np.concatenate([mu, mu.conj()])
    assert np.allclose(np.sort_complex(np.round(ev, 10)), np.sort_complex(np.round(want, 10)),
                       atol=1e-9)


def test_observed_rate_approaches_spectral_radius():
    """Remark 1: with FP64 and tight inner solves, the asymptotic contraction
    of the error equals rho(T_F)."""
    p, xt = conv_diff_2d(8, 74, ny=8)
    orc = O.Oracle(p)
    A, M, N = orc.dense(O.OP_A), orc.dense(O.OP_M), orc.dense(O.OP_N)
    b = orc.rhs(xt)
    alpha, omega = 0.9, 1.0
    rho = max(abs(np.linalg.eigvals(O.iteration_matrix(A, M, N, alpha, omega))))
    x, st = orc.gadi(b, alpha, omega, O.FP64, tol=1e-13, maxit=400, tol_h=1e-14, tol_s=1e-14,
                     inner_stag=0, outer_stag_window=0)
    h = st["history"]
    k = len(h) - 1
    rate = (h[k - 1] / h[k - 21]) ** (1 / 20)
    assert abs(rate - rho) < 0.02 * rho + 1e-3, (rate, rho)


# --------------------------------------------------------------------------
# mixed precision: limiting accuracy (Theorems 2-3, eq. 3.29)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [O.FP64, O.FP32, O.BF16])
def test_mixed_precision_reaches_fp64_accuracy(prec):
    p, xt = conv_diff_2d(16, 81)
    orc = O.Oracle(p)
    A = orc.dense(O.OP_A)
    b = orc.rhs(xt)
    alpha = 2 * alpha_star(p)
    tolh = {O.FP64: 1e-3, O.FP32: 1e-3, O.BF16: 1e-2}[prec]
    x, st = orc.gadi(b, alpha, 1.0, prec, tol=1e-10, maxit=3000, tol_h=tolh, tol_s=tolh)
    assert st["status"] == "OK", st["status"]
    r = np.linalg.norm(b - A @ x)
    be = O.backward_error(r, np.linalg.norm(A, 2), x, b)
    assert be <= 1e-10
    xd = np.linalg.solve(A, b)
    kap = np.linalg.cond(A)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 10 * kap * 1e-10


def test_norm_power_iteration_lower_bound():
    p, xt = conv_diff_2d(9, 82)
    orc = O.Oracle(p)
    A = orc.dense(O.OP_A)
    est = O.norm2_power(lambda v: A @ v, lambda v: A.T @ v, A.shape[0], iters=200)
    true = np.linalg.norm(A, 2)
    assert est <= true * (1 + 1e-12) and est >= 0.999 * true


def test_config1_trajectory_is_monotone_and_capped():
    """Config 1 (64 x 64, alpha 0.5, omega 1, maxit 500, plain FP64): the run
    ends at the iteration cap without reaching 1e-10 (needs ~626 iterations)."""
    from workloads import config1
    p, xt, c = config1()
    orc = O.Oracle(p)
    b = orc.rhs(xt)
    x, st = orc.gadi(b, c["alpha"], c["omega"], O.FP64, tol=c["tol"], maxit=c["maxit"])
    assert st["outer_its"] == 500 and st["status"] == "NOT_CONVERGED"
    h = st["history"]
    assert 1e-9 < h[-1] < 1e-7
    assert np.all(np.diff(h[50:]) < 0)


def _tridiag(n, sub, diag, sup):
    return np.diag(np.full(n, diag)) + np.diag(np.full(n - 1, sub), -1) + np.diag(np.full(n - 1, sup), 1)


@pytest.mark.parametrize("n", [1, 3, 6])
def test_paper_2d_instance_equals_printed_kronecker_form(n):
    """Sec. 5.2's matrix as printed: A = I (x) T + T (x) I, T = Tridiag(-1,2,-1)
    + 2r Tridiag(0.5,0,-0.5) + 100/(n+1)^2 I (Tridiag(sub, diag, super)), r = 1;
    the workload's (beta, kappa) parametrisation must give exactly it."""
    from workloads import paper_cdr_2d
    p, x1 = paper_cdr_2d(n)
    h2 = 1.0 / (n + 1) ** 2
    T = _tridiag(n, -1.0, 2.0, -1.0) + 2.0 * _tridiag(n, 0.5, 0.0, -0.5) + 100.0 * h2 * np.eye(n)
    K = np.kron(np.eye(n), T) + np.kron(T, np.eye(n))
    orc = O.Oracle(p)
    assert np.allclose(orc.dense(O.OP_A), K, rtol=0, atol=1e-14)
    assert np.array_equal(x1, np.ones(n * n))
    M = orc.dense(O.OP_M)
    assert np.allclose(M, (K + K.T) / 2, atol=1e-14)
    assert np.all(np.linalg.eigvalsh(M) > 0)  # M positive definite (Lemma 1's assumption)


@pytest.mark.parametrize("n", [1, 3, 5])
def test_paper_3d_instance_equals_seven_point_kronecker_form(n):
    """Sec. 5.3's matrix with T_x = T_y = T_z = Tridiag(-1-r, 2, -1+r), r = 1/(2n+2)
    (the standard 7-point stencil: our reading of the printed diagonal)."""
    from workloads import paper_cd_3d
    p, _ = paper_cd_3d(n)
    r = 1.0 / (2 * n + 2)
    T = _tridiag(n, -1.0 - r, 2.0, -1.0 + r)
    I = np.eye(n)
    K = np.kron(T, np.kron(I, I)) + np.kron(I, np.kron(T, I)) + np.kron(I, np.kron(I, T))
    assert np.allclose(O.Oracle(p).dense(O.OP_A), K, rtol=0, atol=1e-14)


def test_reaction_term_shifts_the_spectrum():
    """kappa adds kappa I to M (and A) for the real stencil classes."""
    p0, _ = conv_diff_2d(5, 41, beta=(3.0, 1.0), ny=4)
    p1, _ = conv_diff_2d(5, 41, beta=(3.0, 1.0), ny=4)
    p1.kappa = 0.75
    d0, d1 = O.Oracle(p0).dense(O.OP_M), O.Oracle(p1).dense(O.OP_M)
    assert np.allclose(d1 - d0, 0.75 * np.eye(20), rtol=0, atol=1e-15)
    assert np.array_equal(O.Oracle(p1).dense(O.OP_N), O.Oracle(p0).dense(O.OP_N))


def test_paper_complex_instance_equals_printed_form():
    """Sec. 5.4's system -nu Lap w + i V w = f: (nu/h^2) G + i diag(V) with G
    the 5-point graph Laplacian, V = s U[0,1) per point, nu = 1e-5 (64/n)^2.
    The workload is that matrix times h^2/nu; its real block form [[L, -V],
    [V, L]] (interleaved here) has M = L symmetric and N skew."""
    from workloads import paper_complex_rd
    n = 6
    p, w1 = paper_complex_rd(n, seed=9)
    h = 1.0 / (n + 1)
    nu = 1e-5 * (64.0 / n) ** 2
    V = 1e4 * SplitMix64(9).uniform_array(n * n)
    G = np.kron(np.eye(n), _tri(n, -1, 2, -1)) + np.kron(_tri(n, -1, 2, -1), np.eye(n))
    Ap = (nu / h ** 2) * G + 1j * np.diag(V)
    orc = O.Oracle(p)
    g = SplitMix64(10)
    x = g.uniform_array(2 * n * n) - 0.5
    xc = x[0::2] + 1j * x[1::2]
    y = orc.apply(O.OP_A, x)
    yc = (h ** 2 / nu) * (Ap @ xc)
    scale = np.max(np.abs(yc))
    assert np.allclose(y[0::2], yc.real, rtol=0, atol=1e-13 * scale)
    assert np.allclose(y[1::2], yc.imag, rtol=0, atol=1e-13 * scale)
    M, N = orc.dense(O.OP_M), orc.dense(O.OP_N)
    assert np.array_equal(M, M.T) and np.array_equal(N, -N.T)
    assert np.array_equal(M + N, orc.dense(O.OP_A))
    assert np.array_equal(w1, np.ones(2 * n * n))


@pytest.mark.parametrize("prec", [O.FP64, O.FP32, O.BF16])
def test_pointwise_s_solve_per_point_diagonal(prec):
    """S = alpha I + i diag(T_i): the pointwise solve equals the exact complex
    division by (alpha + i fl_s(T_i)), point by point, up to u_s."""
    from workloads import paper_complex_rd
    p, _ = paper_complex_rd(5, seed=11)
    orc = O.Oracle(p)
    g = SplitMix64(12)
    z = np.array([O.round_prec(prec, v) for v in g.uniform_array(2 * p.npoints) - 0.5])
    alpha, omega = 3.0, 0.5
    y, its = orc.solve_s(alpha, omega, prec, z, 1e-3, 100, 10, pointwise=True)
    assert its == 1
    gam = (2 - omega) * alpha
    T = np.array([O.round_prec(prec, t) for t in p.sigma_pt])
    a = O.round_prec(prec, alpha)
    zc = z[0::2] + 1j * z[1::2]
    want = np.array([O.round_prec(prec, O.round_prec(prec, gam) * v) for v in z])
    want = (want[0::2] + 1j * want[1::2]) / (a + 1j * T)
    u = {O.FP64: 2.0 ** -52, O.FP32: 2.0 ** -23, O.BF16: 2.0 ** -7}[prec]
    assert np.allclose(y[0::2] + 1j * y[1::2], want, rtol=0, atol=8 * u * np.max(np.abs(want)))
