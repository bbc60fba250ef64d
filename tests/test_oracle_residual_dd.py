"""Pins of the oracle's double-FP64 residual (u_r about u^2, Sec. 3.1 allows
any u_r <= u): against exact rational arithmetic, against brute-force
rounding of the pair to u_s, and against the forward-error limit of Sec. 3
(with u_r = u the limiting forward error grows like kappa(A) u_r; with
u_r ~ u^2 it is about u)."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from workloads import K_CSR, Problem, SplitMix64, complex_rd, conv_diff_2d, conv_diff_3d, random_csr

FP64, FP32, BF16 = O.FP64, O.FP32, O.BF16


def _float32_neighbours(v: Fraction):
    """The two binary32 numbers around the exact value v (normal range)."""
    f = np.float32(float(v))
    lo_, hi_ = (f, np.nextafter(f, np.float32(np.inf))) if Fraction(float(f)) <= v else \
        (np.nextafter(f, np.float32(-np.inf)), f)
    return lo_, hi_


def _round_exact(v: Fraction, sig: int) -> float:
    """v rounded to the nearest number with `sig` significant bits, ties to
    even (normal binary32 range), by exact rational comparison."""
    if v == 0:
        return 0.0
    s = -1 if v < 0 else 1
    a = abs(v)
    e = math.floor(math.log2(a))
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    q = e - (sig - 1)                      # spacing 2^q in [2^e, 2^(e+1))
    k = a / Fraction(2) ** q
    fl = k.numerator // k.denominator
    fr = k - fl
    if fr > Fraction(1, 2) or (fr == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    r = fl * Fraction(2) ** q
    return s * (math.inf if r >= Fraction(2) ** 128 else float(r))


def _pairs(seed, n=400):
    g = SplitMix64(seed)
    out = []
    for _ in range(n):
        hi = (2 * g.uniform() - 1) * 2.0 ** (int(g.uniform() * 200) - 100)
        lo = (2 * g.uniform() - 1) * math.ulp(hi) / 2
        out.append((hi, lo))
    return out


@pytest.mark.parametrize("prec,sig", [(FP32, 24), (BF16, 8)])
def test_round_pair_equals_exact_rounding(prec, sig):
    cases = _pairs(31 + prec)
    # exact ties of hi at the cut, with lo of either sign and zero
    g = SplitMix64(41 + prec)
    for _ in range(100):
        e = int(g.uniform() * 200) - 100
        k = (1 << (sig - 1)) + int(g.uniform() * ((1 << (sig - 1)) - 1))
        hi = (k + 0.5) * 2.0 ** (e - (sig - 1))
        for s in (1, -1):
            for lo in (math.ulp(hi) / 4, -math.ulp(hi) / 4, 0.0):
                cases.append((s * hi, s * lo))
    # the top of the range: ties that round to infinity or to the largest finite value
    top = (2 - 2.0 ** -(sig - 1)) * 2.0 ** 127
    tie = top + 2.0 ** (127 - sig)
    q = math.ulp(tie) / 4
    cases += [(tie, 0.0), (tie, -q), (tie, q), (-tie, -q), (-tie, q)]
    for hi, lo in cases:
        want = _round_exact(Fraction(hi) + Fraction(lo), sig)
        assert O.round_pair(prec, hi, lo) == want, (hi, lo)
    # FP64: the pair's high part; outside the normal binary32 range: hi rounded
    assert O.round_pair(FP64, 1.0, 1e-20) == 1.0
    assert O.round_pair(FP32, 2.0 ** -140 * 1.5, 1e-60) == O.round_prec(FP32, 2.0 ** -140 * 1.5)


def _exact_residual(orc, p, b, x):
    """r = b - A x in exact rational arithmetic (A's FP64 entries as given)."""
    if p.kind == K_CSR:
        rp, cl, av = p.rowptr, p.col, p.val
        return [Fraction(b[i]) - sum((Fraction(av[k]) * Fraction(x[cl[k]]) for k in range(rp[i], rp[i + 1])),
                                     Fraction(0)) for i in range(len(rp) - 1)]
    A = orc.dense(O.OP_A)  # entries are the stencil coefficients exactly (products with unit vectors)
    out = []
    for i in range(len(b)):
        s = Fraction(b[i])
        for j in np.nonzero(A[i])[0]:
            s -= Fraction(A[i, j]) * Fraction(x[j])
        out.append(s)
    return out


def _small_cases():
    return [conv_diff_2d(6, 301, ny=5), conv_diff_3d(3, 302), complex_rd(4, 303), random_csr(40, 304)]


@pytest.mark.parametrize("case", range(4))
def test_residual_dd_within_dot2_bound(case):
    p, xt = _small_cases()[case]
    orc = O.Oracle(p)
    g = SplitMix64(500 + case)
    x = np.array([g.uniform() for _ in range(p.nvec)])
    # b close to A x so that the residual cancels heavily
    b = orc.rhs(x) + np.array([(2 * g.uniform() - 1) * 1e-9 for _ in range(p.nvec)])
    y = np.array([(2 * g.uniform() - 1) * 1e-7 for _ in range(p.nvec)])
    xo, rh, rl, rs, nrm = orc.residual_dd(FP32, b, x, y)
    assert np.array_equal(xo, x + y)
    ex = _exact_residual(orc, p, b, xo)
    A = orc.dense(O.OP_A) if p.kind != K_CSR else None
    for i, e in enumerate(ex):
        if A is not None:
            mag = abs(b[i]) + sum(abs(A[i, j] * xo[j]) for j in np.nonzero(A[i])[0])
        else:
            mag = abs(b[i]) + sum(abs(p.val[k] * xo[p.col[k]]) for k in range(p.rowptr[i], p.rowptr[i + 1]))
        # Dot2 (Ogita, Rump & Oishi 2005): |hi + lo - r| <= gamma_n^2 sum |terms| (+ tiny)
        assert abs(Fraction(rh[i]) + Fraction(rl[i]) - e) <= Fraction(mag) * Fraction(2) ** -100, i
        assert abs(rl[i]) <= math.ulp(rh[i]) / 2 + 0.0
        assert rs[i] == _round_exact(e, 24), i
    assert nrm == pytest.approx(math.sqrt(sum(float(e) ** 2 for e in ex)), rel=1e-14)


def _cd1d(n, c, seed):
    """1D convection-diffusion tridiag(-1-c, 2, -1+c) as CSR, x_true ~ U[0,1)."""
    rp, col, val = [0], [], []
    for i in range(n):
        if i > 0:
            col.append(i - 1); val.append(-1.0 - c)
        col.append(i); val.append(2.0)
        if i < n - 1:
            col.append(i + 1); val.append(-1.0 + c)
        rp.append(len(col))
    p = Problem(K_CSR, n, rowptr=np.array(rp, np.int32), col=np.array(col, np.int32), val=np.array(val))
    return p, SplitMix64(seed).uniform_array(n)


def reference_solution(p, b):
    """The solution of A x = b to about u: LU solves refined with the exact
    (rational) residual."""
    n = p.npoints
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(p.rowptr[i], p.rowptr[i + 1]):
            A[i, p.col[k]] = p.val[k]
    x = np.linalg.solve(A, b)
    for _ in range(4):
        r = [Fraction(b[i]) - sum(Fraction(p.val[k]) * Fraction(x[p.col[k]])
                                  for k in range(p.rowptr[i], p.rowptr[i + 1])) for i in range(n)]
        x = x + np.linalg.solve(A, np.array([float(v) for v in r]))
    return x


def forward_error_case():
    p, xt = _cd1d(200, 0.3, 5)
    lmin, lmax = 4 * math.sin(math.pi / 402) ** 2, 4 * math.cos(math.pi / 402) ** 2
    return p, xt, math.sqrt(lmin * lmax)


def test_double_fp64_residual_limits_forward_error():
    """Sec. 3: the limiting forward error of mixed-precision GADI is about
    u + kappa(A) u_r; with u_r = u it grows with kappa(A), with u_r ~ u^2 it
    stays at about u.  Run to stagnation (tol 0) with FP32 inner solves."""
    p, xt, alpha = forward_error_case()
    orc = O.Oracle(p)
    b = orc.rhs(xt)
    xref = reference_solution(p, b)
    fe = {}
    for dd in (False, True):
        x, st = orc.gadi(b, alpha, 0.0, FP32, tol=0.0, maxit=20000, tol_h=1e-4, tol_s=1e-4,
                         outer_stag_window=200, residual_dd=dd)
        assert st["status"] == "STAGNATED"
        fe[dd] = np.linalg.norm(x - xref) / np.linalg.norm(xref)
    assert fe[True] <= 4 * 2.0 ** -53, fe
    assert fe[False] >= 4 * fe[True], fe
