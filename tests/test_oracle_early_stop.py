"""Pins of the oracle's early-stop rules (CPU only).

Sec. 5.1 names an early stop for the inner solves and the outer iteration
without defining it; the readings taken are:
  * inner (CG on H, CGNR on S): stop once the recurrence residual has gone
    `stag` consecutive iterations without reaching a new minimum;
  * outer: DIVERGED as soon as relres_k = ||b - A x_k|| / ||b - A x_0|| is
    not finite or exceeds 1e6.

Neither is pinned by comparing the oracle with itself:
  * the inner rule is checked on constructed systems whose residual sequence
    is computed here in exact rational arithmetic (Python fractions: the
    exact CG the FP64 and FP32 oracles approximate).  The sequences have long
    non-improving runs with wide margins, so rounding cannot move the stop,
    and the predicted stop index changes with every value of `stag`: an
    off-by-one, a comparison with the previous residual instead of the best
    one, or a reset in the wrong place all fail;
  * the outer rule is checked on A = -a I, where Algorithm 1 has the closed
    form relres_k = |f|^k, f = 1 - (2 - omega) a / (alpha - a) (the inner
    solves are exact on multiples of I), so the first k with relres_k > 1e6
    is known; three factors bracket the threshold between 531441 and
    1419857.  A non-finite initial residual must give DIVERGED at k = 0.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle as O
from workloads import K_CSR, Problem

# H = alpha I + M with M = diag((lam_i - 1) / 1024), alpha = 1/1024:
# eigenvalues lam_i / 1024, right-hand side b_i / 64 (all dyadic: exact in
# binary64 and binary32)
LAM = [6, 62, 787, 1306, 1523, 1763, 1820, 2359, 3570, 3575, 3597, 3786]
RHS = [36, -15, 10, 17, -35, -34, -34, 59, -51, 34, 27, -50]
ALPHA = 1.0 / 1024


def _csr(rows):
    """CSR Problem from a list of {col: value} dicts."""
    rp, cl, vl = [0], [], []
    for r in rows:
        for j in sorted(r):
            cl.append(j)
            vl.append(r[j])
        rp.append(len(cl))
    return Problem(K_CSR, len(rows), rowptr=np.asarray(rp, np.int32), col=np.asarray(cl, np.int32),
                   val=np.asarray(vl, np.float64))


def _cg_exact(apply, b, maxit):
    """Squared recurrence-residual norms of CG in exact arithmetic (Fractions)."""
    n = len(b)
    r, p, beta = list(b), [Fr(0)] * n, Fr(0)
    rr = sum(v * v for v in r)
    out = []
    for j in range(maxit):
        p = [r[i] + beta * p[i] for i in range(n)] if j else list(r)
        q = apply(p)
        pq = sum(p[i] * q[i] for i in range(n))
        a = rr / pq
        r = [r[i] - a * q[i] for i in range(n)]
        rn = sum(v * v for v in r)
        out.append(rn)
        if rn == 0:
            break
        beta, rr = rn / rr, rn
    return rr0_of(b), out


def rr0_of(b):
    return sum(v * v for v in b)


def _stop_index(rr0, seq, stag):
    """Iterations taken under the rule: stop after `stag` consecutive
    iterations without a new minimum of the residual (no stop: None)."""
    best, since = rr0, 0
    for j, rn in enumerate(seq):
        if rn < best:
            best, since = rn, 0
        else:
            since += 1
            if since >= stag:
                return j + 1
    return None


def _margins_ok(rr0, seq, stop):
    """Every comparison up to the stop is decided by at least 0.1 %."""
    best = rr0
    for rn in seq[:stop]:
        if abs(rn - best) < best * Fr(1, 1000):
            return False
        best = min(best, rn)
    return True


def test_exact_cg_sequence_has_long_non_improving_runs():
    lam = [Fr(v, 1024) for v in LAM]
    b = [Fr(v, 64) for v in RHS]
    rr0, seq = _cg_exact(lambda p: [lam[i] * p[i] for i in range(len(p))], b, 12)
    stops = [_stop_index(rr0, seq, s) for s in range(1, 10)]
    # one iteration at a new minimum, then 8 without one, then new minima
    assert stops[:8] == [s + 1 for s in range(1, 9)], stops
    assert stops[8] is None
    assert all(_margins_ok(rr0, seq, st) for st in stops[:8])


@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_inner_cg_stagnation_stop_matches_exact_arithmetic(prec):
    p = _csr([{i: (LAM[i] - 1) / 1024.0} for i in range(len(LAM))])
    orc = O.Oracle(p)
    rs = np.array(RHS, np.float64) / 64.0
    lam = [Fr(v, 1024) for v in LAM]
    rr0, seq = _cg_exact(lambda v: [lam[i] * v[i] for i in range(len(v))], [Fr(v, 64) for v in RHS], 12)
    for stag in range(1, 10):
        want = _stop_index(rr0, seq, stag) or 12
        z, its = orc.solve_h(ALPHA, prec, rs, 0.0, 12, stag)
        assert its == want, (stag, its, want)
    # the rule off (stag = 0): the iteration cap alone
    _, its = orc.solve_h(ALPHA, prec, rs, 0.0, 12, 0)
    assert its == 12


# S = alpha I + N with N skew in 2 x 2 blocks [[0, c], [-c, 0]]: S^T S =
# (alpha^2 + c^2) I on each block, so CGNR runs CG on a known diagonal
# spectrum (each value twice) with right-hand side S^T g, g = (2 - omega) alpha z
SKEW_C = [Fr(v, 64) for v in (3, 20, 36, 45, 66, 69, 80, 85, 88, 91)]
S_ALPHA = Fr(1, 8)
S_Z = [-8, 60, 10, -20, 60, 44, 6, -4, -54, 43, 27, -48, -28, -32, -20, 18, -38, -10, -3, 33]


def _s_problem():
    rows = []
    for k, c in enumerate(SKEW_C):
        i, j = 2 * k, 2 * k + 1
        # A = I + N (the symmetric part I does not enter the S-solve)
        rows.append({i: 1.0, j: float(c)})
        rows.append({j: 1.0, i: -float(c)})
    return _csr(rows)


def _s_exact(g):
    """S^T g and the operator S^T S in exact arithmetic."""
    n = len(g)

    def S(v, sign):  # S v (sign +1) or S^T v (sign -1)
        out = [S_ALPHA * v[i] for i in range(n)]
        for k, c in enumerate(SKEW_C):
            i, j = 2 * k, 2 * k + 1
            out[i] += sign * c * v[j]
            out[j] -= sign * c * v[i]
        return out

    return S(g, -1), (lambda p: S(S(p, 1), -1))


@pytest.mark.parametrize("prec", [O.FP64, O.FP32])
def test_inner_cgnr_stagnation_stop_matches_exact_arithmetic(prec):
    omega = 1.0
    g = [(2 - Fr(omega)) * S_ALPHA * Fr(v, 64) for v in S_Z]
    t0, op = _s_exact(g)
    rr0, seq = _cg_exact(op, t0, 11)
    stops = {s: _stop_index(rr0, seq, s) for s in range(1, 8)}
    # new minima for 4 iterations, then no new minimum for 5
    assert stops == {1: 5, 2: 6, 3: 7, 4: 8, 5: 9, 6: None, 7: None}, stops
    assert all(_margins_ok(rr0, seq, v) for v in stops.values() if v)
    orc = O.Oracle(_s_problem())
    z = np.array(S_Z, np.float64) / 64.0
    for stag, want in stops.items():
        _, its = orc.solve_s(float(S_ALPHA), omega, prec, z, 0.0, 10, stag)
        assert its == (want or 10), (stag, its, want)


def _neg_identity(n, a):
    return _csr([{i: -a} for i in range(n)])


@pytest.mark.parametrize("m,omega,k_div", [(1, 0.0, 9), (2, 0.0, 7), (3, 0.0, 5)])
def test_outer_diverged_rule_matches_closed_form(m, omega, k_div):
    """A = -a I, a = 1 + 2^-m, alpha = 1: H = -2^-m I and S = I are solved
    exactly, and relres_k = |f|^k with f = 1 - (2 - omega)(1 + 2^m)."""
    a = 1.0 + 2.0 ** -m
    f = 1.0 - (2.0 - omega) * (1.0 + 2.0 ** m)
    ks = [k for k in range(40) if abs(f) ** k > 1e6]
    assert ks[0] == k_div
    p = _neg_identity(4, a)
    orc = O.Oracle(p)
    b = np.array([1.0, -2.0, 0.5, 3.0])
    x, st = orc.gadi(b, 1.0, omega, O.FP64, tol=1e-10, maxit=50, outer_stag_window=0)
    assert st["status"] == "DIVERGED" and st["outer_its"] == k_div, st
    hist = st["history"]
    for k in range(k_div + 1):
        assert abs(hist[k] - abs(f) ** k) <= 1e-9 * abs(f) ** k, (k, hist[k])
    # the same run with a cap below the divergence index is NOT_CONVERGED
    _, st2 = orc.gadi(b, 1.0, omega, O.FP64, tol=1e-10, maxit=k_div - 1, outer_stag_window=0)
    assert st2["status"] == "NOT_CONVERGED" and st2["outer_its"] == k_div - 1


@pytest.mark.parametrize("window,status,its", [(50, "STAGNATED", 50), (51, "NOT_CONVERGED", 200)])
def test_outer_stagnation_rule_matches_closed_form(window, status, its):
    """A = I, alpha = 1: H = 2 I and S = I are solved exactly and relres_k =
    f^k with f = omega / 2 = 1 - 13 * 2^-16, so relres falls by the factor
    f^W over any W iterations: f^50 = 0.99013 (less than a 1 % drop: STAGNATED
    at k = 50 with the 50-iteration window) and f^51 = 0.98994 (never
    stagnates with a 51-iteration window)."""
    f = 1.0 - 13.0 * 2.0 ** -16
    assert f ** 50 > 0.99 > f ** 51
    p = _csr([{i: 1.0} for i in range(4)])
    orc = O.Oracle(p)
    b = np.array([1.0, -2.0, 0.5, 3.0])
    _, st = orc.gadi(b, 1.0, 2.0 * f, O.FP64, tol=1e-10, maxit=200, outer_stag_window=window)
    assert st["status"] == status and st["outer_its"] == its, st
    k = np.arange(its + 1)
    assert np.allclose(st["history"], f ** k, rtol=1e-12)


def test_outer_diverged_on_non_finite_initial_residual():
    """x_0 with an infinite entry makes ||b - A x_0|| infinite, so relres_0 =
    inf / inf is NaN: DIVERGED at k = 0, not OK and not a run to the cap."""
    p = _neg_identity(4, 2.0)
    orc = O.Oracle(p)
    b = np.ones(4)
    x0 = np.array([np.inf, 0.0, 0.0, 0.0])
    _, st = orc.gadi(b, 1.0, 1.0, O.FP64, tol=1e-10, maxit=20, x0=x0, outer_stag_window=0)
    assert st["status"] == "DIVERGED" and st["outer_its"] == 0, st
