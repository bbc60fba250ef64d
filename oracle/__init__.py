"""CPU oracle for three-precision GADI (arXiv 2512.21164) -- TEST INFRASTRUCTURE.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The product path (the CUDA library under
`paper_2512_21164_gb300/` and its binding) never does, and shares no code with
it.

The arithmetic lives in `gadi_oracle.c` (plain C, FP64, FP32 by C float,
BF16 by explicit round-to-nearest-even); this module compiles it with gcc,
loads it with ctypes and adds the library-routine pieces written in NumPy /
SciPy: the HSS splitting of a CSR matrix (M = (A + A^T)/2, N = (A - A^T)/2,
Sec. 5.2), dense matrices for tiny problems, the GADI iteration matrix T_F
(Sec. 2.1), the normwise backward error of eq. (3.2) with ||A||_2 from power
iteration, and closed forms used as pins.

Parity status: every function here is pinned by `tests/test_oracle_*.py`
against closed forms, dense direct solves, invariants or brute force.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gadi_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
# the same source built with -fopenmp: the all-core CPU baseline only (its
# sums are split by thread); parity tests use the sequential build above
_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}

FP64, FP32, BF16 = 0, 1, 2
K_2D5, K_3D7, K_C2D5, K_CSR = 0, 1, 2, 3
OP_A, OP_M, OP_N = 0, 1, 2
STATUS = {0: "OK", 1: "NOT_CONVERGED", 2: "STAGNATED", 3: "DIVERGED"}
_FLAGS = ["-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def _compile(out, extra):
    if os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *_FLAGS, *extra, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build/liboracle.so (gcc, no FMA
    contraction, no OpenMP) and, where gcc has OpenMP, the all-core variant
    liboracle_omp.so used only to time the CPU baseline."""
    os.makedirs(_BUILD, exist_ok=True)
    if force:
        for f in (_LIB, _LIB_OMP):
            if os.path.exists(f):
                os.remove(f)
    _compile(_LIB, [])
    try:
        _compile(_LIB_OMP, ["-fopenmp"])
    except (subprocess.CalledProcessError, OSError):
        pass  # no OpenMP here: the all-core baseline is reported as unavailable
    return _LIB


def has_openmp() -> bool:
    build()
    return os.path.exists(_LIB_OMP)


class _Problem(C.Structure):
    _fields_ = [("kind", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("h", C.c_double), ("beta", C.c_double * 3), ("kappa", C.c_double),
                ("sigma", C.c_double), ("n", C.c_int),
                ("rowptr", C.POINTER(C.c_int)), ("col", C.POINTER(C.c_int)),
                ("aval", C.POINTER(C.c_double)),
                ("mrowptr", C.POINTER(C.c_int)), ("mcol", C.POINTER(C.c_int)),
                ("mval", C.POINTER(C.c_double)), ("nval", C.POINTER(C.c_double)),
                ("sigma_pt", C.POINTER(C.c_double))]


class _Opts(C.Structure):
    _fields_ = [("tol_h", C.c_double), ("tol_s", C.c_double), ("maxit_inner", C.c_int),
                ("inner_stag", C.c_int), ("outer_stag_window", C.c_int),
                ("s_pointwise", C.c_int), ("ur_dd", C.c_int)]


class _Stats(C.Structure):
    _fields_ = [("outer_its", C.c_int), ("inner_h", C.c_long), ("inner_s", C.c_long),
                ("relres", C.c_double), ("status", C.c_int)]


def lib(omp: bool = False):
    """The loaded oracle library; omp=True: the all-core (OpenMP) build."""
    with _lock:
        if omp not in _libs:
            build()
            path = _LIB_OMP if omp else _LIB
            if not os.path.exists(path):
                raise RuntimeError("the OpenMP build of the oracle is unavailable (gcc without -fopenmp)")
            L = C.CDLL(path)
            dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
            pp = C.POINTER(_Problem)
            L.orc_round_bf16.restype = C.c_double
            L.orc_round_bf16.argtypes = [C.c_double]
            L.orc_round.restype = C.c_double
            L.orc_round.argtypes = [C.c_int, C.c_double]
            L.orc_stencil_coeffs.argtypes = [C.c_int, C.c_int, C.c_double, dp, C.c_double,
                                             C.c_double, dp]
            L.orc_stencil_apply.argtypes = [C.c_int] * 4 + [dp, dp, dp]
            L.orc_csr_apply.argtypes = [C.c_int, ip, ip, dp, C.c_double, dp, dp]
            L.orc_apply.argtypes = [pp, C.c_int, dp, dp]
            L.orc_residual.restype = C.c_double
            L.orc_residual.argtypes = [pp, C.c_int, dp, dp, dp, dp, dp, dp]
            L.orc_residual_dd.restype = C.c_double
            L.orc_residual_dd.argtypes = [pp, C.c_int, dp, dp, dp, dp, dp, dp, dp]
            L.orc_round_pair.restype = C.c_double
            L.orc_round_pair.argtypes = [C.c_int, C.c_double, C.c_double]
            L.orc_solve_h.restype = C.c_int
            L.orc_solve_h.argtypes = [pp, C.c_double, C.c_int, dp, dp, C.c_double, C.c_int,
                                      C.c_int]
            L.orc_solve_s.restype = C.c_int
            L.orc_solve_s.argtypes = [pp, C.c_double, C.c_double, C.c_int, dp, dp, C.c_double,
                                      C.c_int, C.c_int, C.c_int]
            L.orc_gadi.restype = C.c_int
            L.orc_gadi.argtypes = [pp, dp, dp, C.c_double, C.c_double, C.c_int, C.c_double,
                                   C.c_int, C.POINTER(_Opts), C.POINTER(_Stats), dp]
            _libs[omp] = L
    return _libs[omp]


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# HSS splitting of a CSR matrix (Sec. 5.2: H = alpha I + (A + A^T)/2,
# S = alpha I + (A - A^T)/2).  scipy.sparse does the transpose and the sums.
# --------------------------------------------------------------------------
def csr_split(rowptr, col, val):
    """Return (mrowptr, mcol, mval, nval): M = (A + A^T)/2 and N = (A - A^T)/2 on
    the common pattern of A + A^T plus the full diagonal, sorted by column."""
    import scipy.sparse as sp
    n = len(rowptr) - 1
    A = sp.csr_matrix((np.asarray(val, np.float64), np.asarray(col), np.asarray(rowptr)),
                      shape=(n, n))
    pat = (abs(A) + abs(A.T) + sp.identity(n, format="csr")).tocsr()
    pat.sort_indices()
    M = ((A + A.T) * 0.5).tocsr()
    N = ((A - A.T) * 0.5).tocsr()
    mrowptr = pat.indptr.astype(np.int32)
    mcol = pat.indices.astype(np.int32)
    rows = np.repeat(np.arange(n), np.diff(pat.indptr))
    mval = np.asarray(M[rows, mcol]).ravel().astype(np.float64)
    nval = np.asarray(N[rows, mcol]).ravel().astype(np.float64)
    return mrowptr, mcol, mval, nval


class Oracle:
    """Bound oracle for one problem (workloads.Problem)."""

    def __init__(self, prob, omp: bool = False):
        self.prob = prob
        self.L = lib(omp)
        self._keep = []
        P = _Problem()
        P.kind, P.nx, P.ny, P.nz = prob.kind, prob.nx, prob.ny, prob.nz
        P.h = prob.hh
        P.beta = (C.c_double * 3)(*prob.beta)
        P.kappa, P.sigma = prob.kappa, prob.sigma
        if prob.kind == K_CSR:
            rp = np.ascontiguousarray(prob.rowptr, np.int32)
            cl = np.ascontiguousarray(prob.col, np.int32)
            av = _f64(prob.val)
            mrp, mcl, mv, nv = csr_split(rp, cl, av)
            self._keep += [rp, cl, av, mrp, mcl, mv, nv]
            P.n = len(rp) - 1
            P.rowptr, P.col, P.aval = _ip(rp), _ip(cl), _dp(av)
            P.mrowptr, P.mcol, P.mval, P.nval = _ip(mrp), _ip(mcl), _dp(mv), _dp(nv)
            self.split = (mrp, mcl, mv, nv)
        else:
            P.n = prob.npoints
            sig = getattr(prob, "sigma_pt", None)
            if prob.kind == K_C2D5 and sig is not None:
                sg = _f64(sig)
                self._keep.append(sg)
                P.sigma_pt = _dp(sg)
        self.P = P
        self.m = prob.nvec

    # -- operators (FP64) --------------------------------------------------
    def apply(self, which, x):
        x = _f64(x)
        y = np.empty(self.m)
        self.L.orc_apply(C.byref(self.P), which, _dp(x), _dp(y))
        return y

    def rhs(self, x_true):
        """b = A x_true in FP64 (the oracle's own operator)."""
        return self.apply(OP_A, x_true)

    def coeffs(self, part):
        out = np.zeros(8)
        b = (C.c_double * 3)(*self.prob.beta)
        self.L.orc_stencil_coeffs(self.prob.kind, part, self.prob.hh, b, self.prob.kappa,
                                 self.prob.sigma, _dp(out))
        return out

    # -- steps of Algorithm 1 ---------------------------------------------
    def residual(self, prec, b, x, y=None):
        """(x_out, r, r_s, ||r||): x_out = x + y, r = b - A x_out (FP64), r_s = fl_s(r)."""
        b, x = _f64(b), _f64(x)
        yy = _f64(y) if y is not None else None
        xo, r, rs = np.empty(self.m), np.empty(self.m), np.empty(self.m)
        nrm = self.L.orc_residual(C.byref(self.P), prec, _dp(b), _dp(x),
                                 _dp(yy) if yy is not None else None, _dp(xo), _dp(r), _dp(rs))
        return xo, r, rs, nrm

    def residual_dd(self, prec, b, x, y=None):
        """(x_out, r_hi, r_lo, r_s, ||r_hi||): the residual in double-FP64 (u_r
        about u^2), r = r_hi + r_lo, r_s = the pair rounded to u_s."""
        b, x = _f64(b), _f64(x)
        yy = _f64(y) if y is not None else None
        xo, rh, rl, rs = (np.empty(self.m) for _ in range(4))
        nrm = self.L.orc_residual_dd(C.byref(self.P), prec, _dp(b), _dp(x),
                                    _dp(yy) if yy is not None else None, _dp(xo), _dp(rh), _dp(rl),
                                    _dp(rs))
        return xo, rh, rl, rs, nrm

    def solve_h(self, alpha, prec, rs, tol, maxit=1000, stag=10):
        rs = _f64(rs)
        z = np.empty(self.m)
        its = self.L.orc_solve_h(C.byref(self.P), alpha, prec, _dp(rs), _dp(z), tol, maxit, stag)
        return z, its

    def solve_s(self, alpha, omega, prec, z, tol, maxit=1000, stag=10, pointwise=False):
        z = _f64(z)
        y = np.empty(self.m)
        its = self.L.orc_solve_s(C.byref(self.P), alpha, omega, prec, _dp(z), _dp(y), tol, maxit,
                                stag, int(pointwise))
        return y, its

    def gadi(self, b, alpha, omega, prec, tol=1e-10, maxit=500, x0=None, tol_h=1e-3,
             tol_s=1e-3, maxit_inner=1000, inner_stag=10, outer_stag_window=50,
             s_pointwise=False, residual_dd=False):
        """Algorithm 1 (residual_dd: u_r = double-FP64).  Returns (x, stats dict
        with relres history)."""
        b = _f64(b)
        x = np.zeros(self.m) if x0 is None else _f64(x0).copy()
        o = _Opts(tol_h, tol_s, maxit_inner, inner_stag, outer_stag_window, int(s_pointwise),
                  int(residual_dd))
        st = _Stats()
        hist = np.zeros(maxit + 2)
        self.L.orc_gadi(C.byref(self.P), _dp(b), _dp(x), alpha, omega, prec, tol, maxit,
                       C.byref(o), C.byref(st), _dp(hist))
        k = st.outer_its
        return x, dict(outer_its=k, inner_h=st.inner_h, inner_s=st.inner_s, relres=st.relres,
                       status=STATUS[st.status], history=hist[:k + 1].copy())

    # -- dense forms for tiny problems --------------------------------------
    def dense(self, which):
        """Dense matrix of operator `which` (A, M or N) by applying it to unit
        vectors; complex problems give the real 2n x 2n block form."""
        m = self.m
        D = np.zeros((m, m))
        e = np.zeros(m)
        for j in range(m):
            e[:] = 0.0
            e[j] = 1.0
            D[:, j] = self.apply(which, e)
        return D


def round_bf16(v):
    return lib().orc_round_bf16(float(v))


def round_prec(prec, v):
    return lib().orc_round(prec, float(v))


def round_pair(prec, hi, lo):
    """hi + lo rounded to u_s (ties of hi decided by lo in the normal binary32 range)."""
    return lib().orc_round_pair(prec, float(hi), float(lo))


def iteration_matrix(A, M, N, alpha, omega):
    """T_F(alpha, omega) = (alpha I + N)^-1 (alpha I + M)^-1 (alpha^2 I + M N - (1-omega) alpha A)
    (Sec. 2.1), dense."""
    n = A.shape[0]
    I = np.eye(n)
    return np.linalg.solve(alpha * I + N, np.linalg.solve(alpha * I + M,
                           alpha ** 2 * I + M @ N - (1.0 - omega) * alpha * A))


def two_step_gadi(A, M, N, b, alpha, omega, iters, x0=None):
    """The two-step GADI iteration of Sec. 2.1 with dense direct solves:
    (aI + M) x_half = (aI - N) x + b;  (aI + N) x_new = (N - (1-w) a I) x + (2-w) a x_half."""
    n = A.shape[0]
    I = np.eye(n)
    x = np.zeros(n) if x0 is None else x0.copy()
    out = [x.copy()]
    for _ in range(iters):
        xh = np.linalg.solve(alpha * I + M, (alpha * I - N) @ x + b)
        x = np.linalg.solve(alpha * I + N, (N - (1.0 - omega) * alpha * I) @ x
                            + (2.0 - omega) * alpha * xh)
        out.append(x.copy())
    return out


def alg1_dense(A, M, N, b, alpha, omega, iters, x0=None):
    """Algorithm 1 with dense direct subsolves in FP64 (no rounding)."""
    n = A.shape[0]
    I = np.eye(n)
    x = np.zeros(n) if x0 is None else x0.copy()
    out = [x.copy()]
    for _ in range(iters):
        r = b - A @ x
        z = np.linalg.solve(alpha * I + M, r)
        y = np.linalg.solve(alpha * I + N, (2.0 - omega) * alpha * z)
        x = x + y
        out.append(x.copy())
    return out


def norm2_power(apply_A, apply_At, m, iters=50, seed=0):
    """||A||_2 estimate: power iteration on A^T A (a lower bound)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(m)
    v /= np.linalg.norm(v)
    s = 0.0
    for _ in range(iters):
        w = apply_At(apply_A(v))
        s = np.linalg.norm(w)
        if s == 0:
            return 0.0
        v = w / s
    return float(np.sqrt(s))


def backward_error(r_norm, A_norm, x, b):
    """Normwise backward error ||b - A x|| / (||A|| ||x|| + ||b||), eq. (3.2)."""
    return float(r_norm / (A_norm * np.linalg.norm(x) + np.linalg.norm(b)))
