"""Python binding of the GB300 GADI library (include/gadi.h).

Argument marshalling only: every step of the solve runs in the CUDA library
`_build/libgadi.so` (built by `paper_2512_21164_gb300.build`).  Vectors are
torch tensors (CUDA or CPU) or NumPy arrays (host); their raw pointers are
handed to the C ABI, which detects host vs device memory itself.  There is no
CPU fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgadi.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "gadi.h")

# enums of gadi.h
OK, NOT_CONVERGED, STAGNATED, DIVERGED = 0, 1, 2, 3
ERR_INVALID, ERR_NONFINITE, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6
FP64, FP32, BF16 = 0, 1, 2
FP64X2 = 3  # double-FP64: a residual precision (gadi_opts.u_r) only
SPLIT_HSS = 0
STENCIL_2D5, STENCIL_3D7, COMPLEX_2D5, CSR = 0, 1, 2, 3
OP_A, OP_M, OP_N, OP_AT = 0, 1, 2, 3
PREC_NAMES = {"fp64": FP64, "fp32": FP32, "bf16": BF16}


class GadiError(RuntimeError):
    def __init__(self, status: int, what: str):
        detail = ""
        if status in (ERR_CUDA, ERR_OOM):
            detail = " -- " + last_error()
        super().__init__(f"{what}: {status_str(status)} ({status}){detail}")
        self.status = status


class Problem(C.Structure):
    _fields_ = [("kind", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("h", C.c_double), ("beta", C.c_double * 3), ("kappa", C.c_double),
                ("sigma", C.c_double), ("n", C.c_int), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p), ("sigma_pt", C.c_void_p)]


class Opts(C.Structure):
    _fields_ = [("tol_h", C.c_double), ("tol_s", C.c_double), ("maxit_inner", C.c_int),
                ("inner_stag", C.c_int), ("outer_stag_window", C.c_int),
                ("s_pointwise", C.c_int), ("stream", C.c_void_p), ("max_blocks", C.c_int),
                ("hist", C.c_void_p), ("batch_group", C.c_int), ("alpha_restarts", C.c_int),
                ("h_resident", C.c_int), ("u_r", C.c_int), ("s_resident", C.c_int),
                ("backward_err", C.c_int), ("batch_interleave", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("outer_its", C.c_int), ("inner_its_h", C.c_longlong),
                ("inner_its_s", C.c_longlong), ("relres", C.c_double), ("r0_norm", C.c_double),
                ("seconds", C.c_double), ("status", C.c_int), ("blocks", C.c_int),
                ("alpha", C.c_double), ("restarts", C.c_int), ("h_resident", C.c_int),
                ("s_resident", C.c_int), ("backward_err", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lock = threading.Lock()
_L = None


def lib():
    """Load libgadi.so (raises if it has not been built)."""
    global _L
    with _lock:
        if _L is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"GADI CUDA library not built: {LIB_PATH} missing "
                                   "(run paper_2512_21164_gb300.build.build())")
            L = C.CDLL(LIB_PATH)
            vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
            L.gadi_opts_default.argtypes = [C.POINTER(Opts), C.c_int]
            L.gadi_opts_default.restype = None
            L.gadi_status_str.argtypes = [C.c_int]
            L.gadi_status_str.restype = C.c_char_p
            L.gadi_last_error.argtypes = []
            L.gadi_last_error.restype = C.c_char_p
            L.gadi_create.argtypes = [C.POINTER(Problem), C.c_int, C.POINTER(vp)]
            L.gadi_destroy.argtypes = [vp]
            L.gadi_destroy.restype = None
            L.gadi_solve.argtypes = [vp, vp, vp, C.c_double, C.c_double, C.c_int, C.c_int,
                                     C.c_double, C.c_int, C.POINTER(Opts), C.POINTER(Stats)]
            L.gadi_apply.argtypes = [vp, C.c_int, vp, vp, vp]
            L.gadi_norm2_estimate.argtypes = [vp, C.c_int, dp, vp]
            L.gadi_step_residual.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp, vp, dp, vp]
            L.gadi_step_residual_ur.argtypes = [vp, C.c_int, C.c_int, vp, vp, vp, vp, vp, vp, vp, dp, vp]
            L.gadi_step_residual_ur.restype = C.c_int
            L.gadi_step_solve_h.argtypes = [vp, C.c_double, C.c_int, vp, vp, C.c_double, C.c_int,
                                            C.c_int, ip, vp]
            L.gadi_step_solve_s.argtypes = [vp, C.c_double, C.c_double, C.c_int, vp, vp,
                                            C.c_double, C.c_int, C.c_int, C.c_int, ip, vp]
            L.gadi_solve_batched.argtypes = [vp, C.c_int, C.c_int, vp, vp, vp, C.c_double, C.c_int,
                                             C.c_int, C.c_double, C.c_int, C.POINTER(Opts),
                                             C.POINTER(Stats)]
            L.gadi_solve_batched.restype = C.c_int
            L.gadi_condition_numbers.argtypes = [C.POINTER(Problem), C.c_double, dp, dp]
            L.gadi_condition_numbers.restype = C.c_int
            L.gadi_select_alpha.argtypes = [C.POINTER(Problem), C.c_double, C.c_int, C.c_double, dp]
            L.gadi_select_alpha.restype = C.c_int
            L.gadi_selftest_barrier.argtypes = [C.c_int, C.c_double]
            L.gadi_selftest_barrier.restype = C.c_int
            L.gadi_stencil_coefs.argtypes = [C.POINTER(Problem), C.c_int, dp]
            L.gadi_stencil_coefs.restype = C.c_int
            L.gadi_probe_sync.argtypes = [C.c_int, C.c_int, dp]
            L.gadi_probe_sync.restype = C.c_int
            L.gadi_probe_fp64.argtypes = [C.c_int, dp, dp]
            L.gadi_probe_fp64.restype = C.c_int
            L.gadi_selftest_convert.argtypes = [vp, C.c_longlong, C.POINTER(C.c_longlong)]
            L.gadi_selftest_convert.restype = C.c_int
            L.gadi_batch_plan.argtypes = [C.c_int, C.POINTER(C.c_longlong), C.POINTER(C.c_int),
                                          C.POINTER(C.c_double), C.c_int, C.c_int, C.POINTER(C.c_int),
                                          C.POINTER(C.c_int), C.POINTER(C.c_double)]
            L.gadi_batch_plan.restype = C.c_int
            L.gadi_solve_h_2d_noalloc.argtypes = [C.c_int, C.c_int, C.c_double, C.c_int, vp, vp,
                                                  C.c_double, C.c_int, C.c_int, ip, vp]
            for f in ("gadi_create", "gadi_solve", "gadi_apply", "gadi_norm2_estimate",
                      "gadi_step_residual", "gadi_step_solve_h", "gadi_step_solve_s",
                      "gadi_solve_h_2d_noalloc"):
                getattr(L, f).restype = C.c_int
            _L = L
    return _L


def status_str(s: int) -> str:
    return lib().gadi_status_str(int(s)).decode()


def last_error() -> str:
    return lib().gadi_last_error().decode()


def _ptr(a):
    """Raw pointer of a torch tensor or NumPy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, int):  # a raw address
        return a
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported vector type {type(a)}")


def _stream(stream):
    if stream is not None:
        return stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def default_opts(u_low: int) -> Opts:
    o = Opts()
    lib().gadi_opts_default(C.byref(o), u_low)
    return o


class Gadi:
    """One linear system: a handle of the C ABI (gadi_create / gadi_destroy)."""

    def __init__(self, kind, nx=0, ny=1, nz=1, h=0.0, beta=(0.0, 0.0, 0.0), kappa=0.0,
                 sigma=0.0, rowptr=None, col=None, val=None, sigma_pt=None):
        import numpy as np
        P = Problem()
        P.kind, P.nx, P.ny, P.nz, P.h = int(kind), int(nx), int(ny), int(nz), float(h)
        P.beta = (C.c_double * 3)(*[float(b) for b in beta])
        P.kappa, P.sigma = float(kappa), float(sigma)
        self._keep = []
        if kind == CSR:
            rp = np.ascontiguousarray(rowptr, np.int32)
            cl = np.ascontiguousarray(col, np.int32)
            vl = np.ascontiguousarray(val, np.float64)
            self._keep = [rp, cl, vl]
            P.n = len(rp) - 1
            P.rowptr, P.col, P.val = rp.ctypes.data, cl.ctypes.data, vl.ctypes.data
            self.nvec = P.n
        else:
            n = int(nx) * int(ny) * (int(nz) if kind == STENCIL_3D7 else 1)
            self.nvec = 2 * n if kind == COMPLEX_2D5 else n
            if sigma_pt is not None:
                sg = np.ascontiguousarray(sigma_pt, np.float64)
                self._keep = [sg]
                P.sigma_pt = sg.ctypes.data
        self.kind = kind
        h_ = C.c_void_p()
        st = lib().gadi_create(C.byref(P), SPLIT_HSS, C.byref(h_))
        if st != OK:
            raise GadiError(st, "gadi_create")
        self.h = h_

    @classmethod
    def from_problem(cls, p):
        """From a workloads.Problem descriptor."""
        return cls(p.kind, p.nx, p.ny, p.nz, p.h, p.beta, p.kappa, p.sigma, p.rowptr, p.col, p.val,
                   getattr(p, "sigma_pt", None))

    def close(self):
        if getattr(self, "h", None):
            lib().gadi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------------
    def solve(self, b, x, alpha, omega=1.0, u_low=FP32, tol=1e-10, maxit=1000, opts=None,
              hist=None, stream=None, check=True, **kw):
        """gadi_solve: x (in/out) <- Algorithm 1 iterate.  Returns (status, stats dict)."""
        o = default_opts(u_low) if opts is None else opts
        for k, v in kw.items():
            setattr(o, k, v)
        o.stream = _stream(stream)
        if hist is not None:
            o.hist = _ptr(hist)
        s = Stats()
        st = lib().gadi_solve(self.h, _ptr(b), _ptr(x), float(alpha), float(omega), FP64,
                              int(u_low), float(tol), int(maxit), C.byref(o), C.byref(s))
        if check and st < 0:
            raise GadiError(st, "gadi_solve")
        return st, s.as_dict()

    def apply(self, op, x, y, stream=None):
        st = lib().gadi_apply(self.h, int(op), _ptr(x), _ptr(y), _stream(stream))
        if st != OK:
            raise GadiError(st, "gadi_apply")
        return y

    def norm2(self, iters=50, stream=None):
        out = C.c_double()
        st = lib().gadi_norm2_estimate(self.h, int(iters), C.byref(out), _stream(stream))
        if st != OK:
            raise GadiError(st, "gadi_norm2_estimate")
        return out.value

    def step_residual(self, u_low, b, x, y, x_out, r_out, rs, stream=None):
        nrm = C.c_double()
        st = lib().gadi_step_residual(self.h, int(u_low), _ptr(b), _ptr(x), _ptr(y), _ptr(x_out),
                                      _ptr(r_out), _ptr(rs), C.byref(nrm), _stream(stream))
        if st != OK:
            raise GadiError(st, "gadi_step_residual")
        return nrm.value

    def step_residual_ur(self, u_r, u_low, b, x, y, x_out, r_out, r_lo_out, rs, stream=None):
        """gadi_step_residual_ur: the residual step in precision u_r (FP64 or
        FP64X2); returns ||r||."""
        nrm = C.c_double()
        st = lib().gadi_step_residual_ur(self.h, int(u_r), int(u_low), _ptr(b), _ptr(x), _ptr(y),
                                         _ptr(x_out), _ptr(r_out), _ptr(r_lo_out), _ptr(rs),
                                         C.byref(nrm), _stream(stream))
        if st != OK:
            raise GadiError(st, "gadi_step_residual_ur")
        return nrm.value

    def step_solve_h(self, alpha, u_low, rs, z, tol, maxit, stag=0, stream=None):
        its = C.c_int()
        st = lib().gadi_step_solve_h(self.h, float(alpha), int(u_low), _ptr(rs), _ptr(z),
                                     float(tol), int(maxit), int(stag), C.byref(its),
                                     _stream(stream))
        if st != OK:
            raise GadiError(st, "gadi_step_solve_h")
        return its.value

    def step_solve_s(self, alpha, omega, u_low, z, y, tol, maxit, stag=0, pointwise=True,
                     stream=None):
        its = C.c_int()
        st = lib().gadi_step_solve_s(self.h, float(alpha), float(omega), int(u_low), _ptr(z),
                                     _ptr(y), float(tol), int(maxit), int(stag), int(pointwise),
                                     C.byref(its), _stream(stream))
        if st != OK:
            raise GadiError(st, "gadi_step_solve_s")
        return its.value


def selftest_barrier(nblocks=64, timeout_ms=50.0):
    """gadi_selftest_barrier: a grid barrier whose wait runs out; returns the status
    (GADI_ERR_TIMEOUT expected)."""
    return lib().gadi_selftest_barrier(int(nblocks), float(timeout_ms))


def probe_sync(nblocks=0, iters=20000):
    """gadi_probe_sync: mean microseconds of one grid-wide sum of the inner
    solves (two FP32 values, bounded grid barrier) on `nblocks` blocks."""
    out = C.c_double()
    st = lib().gadi_probe_sync(int(nblocks), int(iters), C.byref(out))
    if st != OK:
        raise GadiError(st, "gadi_probe_sync")
    return out.value


def probe_fp64(iters=200000):
    """gadi_probe_fp64: (10^9 FP64 FMA per second, FMA per SM per clock)."""
    g, r = C.c_double(), C.c_double()
    st = lib().gadi_probe_fp64(int(iters), C.byref(g), C.byref(r))
    if st != OK:
        raise GadiError(st, "gadi_probe_fp64")
    return g.value, r.value


# the candidate group sizes of the batched solve's tuner (2^i blocks)
BATCH_SIZES = (1, 2, 4, 8, 16, 32, 64)


def batch_plan(side, count, t_outer=None, fixed=0, total=152):
    """gadi_batch_plan (host only): the batched solve's layout for size classes
    (largest first) with grid sides `side`, unit counts `count` and per-class
    seconds per outer iteration on groups of BATCH_SIZES blocks (`t_outer`,
    ncl x 7; <= 0 = not admitted).  Returns (sizes, groups, estimate)."""
    n = len(side)
    sd = (C.c_longlong * n)(*[int(v) for v in side])
    cn = (C.c_int * n)(*[int(v) for v in count])
    t = None
    if t_outer is not None:
        flat = [float(v) for row in t_outer for v in row]
        if len(flat) != 7 * n:
            raise ValueError("t_outer: 7 timings per class")
        t = (C.c_double * len(flat))(*flat)
    sz, gr, est = (C.c_int * n)(), (C.c_int * n)(), C.c_double()
    st = lib().gadi_batch_plan(n, sd, cn, t, int(fixed), int(total), sz, gr, C.byref(est))
    if st != OK:
        raise GadiError(st, "gadi_batch_plan")
    return list(sz), list(gr), est.value


def selftest_convert(d):
    """gadi_selftest_convert on a device float64 tensor: mismatch counts of the
    integer-pipe conversions (f64->f32, f64->bf16, f32->f64) against the
    hardware ones, and of f32->bf16 by instruction against the integer one."""
    out = (C.c_longlong * 4)()
    st = lib().gadi_selftest_convert(_ptr(d), int(d.numel()), out)
    if st != OK:
        raise GadiError(st, "gadi_selftest_convert")
    return list(out)


def _problem_struct(p):
    P = Problem()
    P.kind, P.nx, P.ny, P.nz, P.h = int(p.kind), int(p.nx), int(p.ny), int(p.nz), float(p.h)
    P.beta = (C.c_double * 3)(*[float(x) for x in p.beta])
    P.kappa, P.sigma = float(p.kappa), float(p.sigma)
    sig = getattr(p, "sigma_pt", None)
    if sig is not None:
        import numpy as np
        sg = np.ascontiguousarray(sig, np.float64)
        P._sig = sg  # keep alive with the struct
        P.sigma_pt = sg.ctypes.data
    return P


def stencil_coefs(p, op=OP_A):
    """gadi_stencil_coefs: [centre, W, E, S, N, B, T, imaginary diagonal] of
    Op for a workloads.Problem of a stencil class."""
    out = (C.c_double * 8)()
    st = lib().gadi_stencil_coefs(C.byref(_problem_struct(p)), int(op), out)
    if st != OK:
        raise GadiError(st, "gadi_stencil_coefs")
    return list(out)


def stencil_csr(p, op=OP_A):
    """The matrix of Op for a real 2D or 3D stencil problem assembled as CSR
    (host NumPy arrays rowptr, col int32, val float64; columns in increasing
    order, zero Dirichlet boundary), from the library's own coefficients."""
    import numpy as np
    if p.kind not in (STENCIL_2D5, STENCIL_3D7):
        raise ValueError("real stencil classes only")
    c = stencil_coefs(p, op)
    nx, ny, nz = p.nx, p.ny, (p.nz if p.kind == STENCIL_3D7 else 1)
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.int64)
    ix, iy, iz = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    # (offset, coefficient, valid mask) in increasing column order
    terms = []
    if p.kind == STENCIL_3D7:
        terms.append((-nx * ny, c[5], iz > 0))
    terms += [(-nx, c[3], iy > 0), (-1, c[1], ix > 0), (0, c[0], np.ones(n, bool)),
              (1, c[2], ix < nx - 1), (nx, c[4], iy < ny - 1)]
    if p.kind == STENCIL_3D7:
        terms.append((nx * ny, c[6], iz < nz - 1))
    mask = np.stack([t[2] for t in terms], axis=1)
    cols = np.stack([idx + t[0] for t in terms], axis=1)
    vals = np.stack([np.full(n, t[1]) for t in terms], axis=1)
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, np.int64)
    rowptr[1:] = np.cumsum(counts)
    return rowptr.astype(np.int32), cols[mask].astype(np.int32), vals[mask].astype(np.float64)


def condition_numbers(p, alpha):
    """gadi_condition_numbers (Sec. 4.3, the condition check of eq. 4.1) for a workloads.Problem: (kappa_H, kappa_S bound)."""
    kh, ks = C.c_double(), C.c_double()
    st = lib().gadi_condition_numbers(C.byref(_problem_struct(p)), float(alpha), C.byref(kh), C.byref(ks))
    if st != OK:
        raise GadiError(st, "gadi_condition_numbers")
    return kh.value, ks.value


def select_alpha(p, alpha0, u_low, tau=0.01):
    """gadi_select_alpha (Sec. 4.3 steps 2-3)."""
    out = C.c_double()
    st = lib().gadi_select_alpha(C.byref(_problem_struct(p)), float(alpha0), int(u_low), float(tau),
                                 C.byref(out))
    if st != OK:
        raise GadiError(st, "gadi_select_alpha")
    return out.value


def solve_batched(systems, nrhs, bs, xs, alphas, omega=1.0, u_low=FP32, tol=1e-10, maxit=1000,
                  opts=None, stream=None, check=True, **kw):
    """gadi_solve_batched: `systems` are Gadi handles of the 2D 5-point class;
    bs[s] / xs[s] are device tensors holding nrhs consecutive vectors of system s
    (x in/out); alphas[s] per system.  Returns (status, list of per-unit stats
    dicts in the order s*nrhs + j)."""
    n = len(systems)
    o = default_opts(u_low) if opts is None else opts
    for k, v in kw.items():
        setattr(o, k, v)
    o.stream = _stream(stream)
    H = (C.c_void_p * n)(*[h.h.value for h in systems])
    B = (C.c_void_p * n)(*[_ptr(t) for t in bs])
    X = (C.c_void_p * n)(*[_ptr(t) for t in xs])
    A = (C.c_double * n)(*[float(a) for a in alphas])
    S = (Stats * (n * nrhs))()
    st = lib().gadi_solve_batched(H, n, int(nrhs), B, X, A, float(omega), FP64, int(u_low), float(tol),
                                  int(maxit), C.byref(o), S)
    if check and st < 0:
        raise GadiError(st, "gadi_solve_batched")
    return st, [S[i].as_dict() for i in range(n * nrhs)]


def solve_h_2d_noalloc(nx, ny, alpha, u_low, rs, z, tol, maxit, stag=0, stream=None, check=True):
    """gadi_solve_h_2d_noalloc: CG on (alpha I + M) z = rs for the 2D 5-point
    class without any device allocation (for callers that cannot allocate;
    the scratch is a static device array, grids up to 262144 points).
    rs and z are device tensors in u_s.  Returns (status, iterations)."""
    its = C.c_int()
    st = lib().gadi_solve_h_2d_noalloc(int(nx), int(ny), float(alpha), int(u_low), _ptr(rs), _ptr(z),
                                       float(tol), int(maxit), int(stag), C.byref(its), _stream(stream))
    if check and st != OK:
        raise GadiError(st, "gadi_solve_h_2d_noalloc")
    return st, its.value


def header_functions(path: str = HEADER) -> list[str]:
    """Names of the functions include/gadi.h declares."""
    import re
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gadi_\w+)\s*\(", src)))
