"""Data-driven choice of the GADI parameter alpha (Sec. 4.2 of arXiv 2512.21164).

Sec. 4.2 trains a Gaussian-process regression (GPR) on small instances of a
problem family and uses it to predict a near-optimal alpha for larger ones;
Sec. 4.3 then checks the condition-number bound and raises alpha on
stagnation (`gadi_select_alpha`, `gadi_opts.alpha_restarts`).  The paper does
not give the features, targets or training set; this module's choices:

* target: log2(alpha_best / alpha_ref), alpha_ref a reference value the
  caller supplies -- typically alpha* = sqrt(lambda_min(M) lambda_max(M)), the
  closed-form HSS optimum of the family's M (the ratio varies slowly with the
  size, alpha itself like 1/n);
* feature: log2 of the grid size n (one GP per problem family, inner
  precision and omega);
* alpha_best on a training size: the swept factor whose solve to the target
  tolerance moves the fewest algorithmic bytes (the byte model of the
  benchmark: outer residual 3d + 2s per point, each inner iteration 8s, the
  CGNR set-up 2s), which is deterministic (iteration counts) and tracks time
  on a bandwidth-bound GPU.

The regression is the standard zero-mean GP with a squared-exponential kernel
plus noise, posterior by Cholesky factorisation (Rasmussen & Williams,
"Gaussian Processes for Machine Learning", MIT Press 2006, Algorithm 2.1), the
targets centred on their mean, the hyperparameters (length scale, signal and
noise standard deviations) chosen by maximising the log marginal likelihood
over a grid.  NumPy only; the sweeps call the library's own solver.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _sqexp(a: np.ndarray, b: np.ndarray, ell: float, sf: float) -> np.ndarray:
    d = a[:, None] - b[None, :]
    return sf * sf * np.exp(-0.5 * (d / ell) ** 2)


def log_marginal_likelihood(x: np.ndarray, y: np.ndarray, ell: float, sf: float, sn: float) -> float:
    """log p(y | x) of a zero-mean GP with kernel sf^2 exp(-(x-x')^2 / (2 ell^2))
    and noise variance sn^2 (Rasmussen & Williams, eq. 2.30)."""
    n = len(x)
    K = _sqexp(x, x, ell, sf) + sn * sn * np.eye(n)
    L = np.linalg.cholesky(K)
    a = np.linalg.solve(L.T, np.linalg.solve(L, y))
    return float(-0.5 * y @ a - np.sum(np.log(np.diag(L))) - 0.5 * n * math.log(2 * math.pi))


@dataclass
class GP1D:
    """A 1D GP regression: fit(x, y), then predict(x*) -> (mean, std)."""

    ell: float = 1.0
    sf: float = 1.0
    sn: float = 0.05
    x: np.ndarray = field(default_factory=lambda: np.zeros(0))
    mu: float = 0.0
    L: np.ndarray | None = None
    a: np.ndarray | None = None

    def fit(self, x, y, ells=None, sfs=None, sns=None):
        x = np.asarray(x, np.float64)
        y = np.asarray(y, np.float64)
        self.x = x
        self.mu = float(np.mean(y)) if len(y) else 0.0
        yc = y - self.mu
        span = float(np.ptp(x)) if len(x) > 1 else 1.0
        ells = ells if ells is not None else span * np.array([0.25, 0.5, 1.0, 2.0, 4.0])
        sy = float(np.std(yc)) if len(yc) > 1 else 1.0
        sfs = sfs if sfs is not None else max(sy, 1e-3) * np.array([0.5, 1.0, 2.0])
        sns = sns if sns is not None else np.array([0.05, 0.1, 0.25, 0.5])
        best = None
        for ell in ells:
            for sf in sfs:
                for sn in sns:
                    lml = log_marginal_likelihood(x, yc, ell, sf, sn)
                    if best is None or lml > best[0]:
                        best = (lml, ell, sf, sn)
        _, self.ell, self.sf, self.sn = best
        K = _sqexp(x, x, self.ell, self.sf) + self.sn ** 2 * np.eye(len(x))
        self.L = np.linalg.cholesky(K)
        self.a = np.linalg.solve(self.L.T, np.linalg.solve(self.L, yc))
        return self

    def predict(self, xs):
        xs = np.atleast_1d(np.asarray(xs, np.float64))
        ks = _sqexp(xs, self.x, self.ell, self.sf)
        mean = self.mu + ks @ self.a
        v = np.linalg.solve(self.L, ks.T)
        var = self.sf ** 2 - np.sum(v * v, axis=0)
        return mean, np.sqrt(np.maximum(var, 0.0))


def solve_bytes(npoints: int, stats: dict, s_bytes: int, d_bytes: int = 8) -> float:
    """Algorithmic bytes of a solve (the benchmark's byte model)."""
    k = stats["outer_its"]
    per_pt = (k + 1) * (3 * d_bytes + 2 * s_bytes) + 8 * s_bytes * (stats["inner_its_h"] + stats["inner_its_s"]) \
        + 2 * s_bytes * k
    return float(npoints) * per_pt


def sweep(family, n: int, prec: int, omega: float, log2_factors, tol: float, alpha_ref, maxit: int = 20000,
          tol_inner: float | None = None):
    """Solve family(n) (a (problem descriptor, x_true) pair; b = A x_true) for
    alpha = 2^f alpha_ref(problem) for each f: [(f, bytes, status)], bytes =
    inf for runs that do not reach tol."""
    import torch

    from . import BF16, COMPLEX_2D5, FP32, FP64, OK, OP_A, Gadi
    p, xt = family(n)
    a0 = alpha_ref(p)
    cplx = p.kind == COMPLEX_2D5
    sb = {FP64: 8, FP32: 4, BF16: 2}[prec] * (2 if cplx else 1)
    db = 16 if cplx else 8
    tin = tol_inner if tol_inner is not None else (1e-2 if prec == BF16 else 1e-3)
    out = []
    with Gadi.from_problem(p) as H:
        xtd = torch.from_numpy(np.ascontiguousarray(xt)).cuda()
        b = torch.zeros_like(xtd)
        H.apply(OP_A, xtd, b)
        x = torch.zeros_like(b)
        for f in log2_factors:
            x.zero_()
            st, s = H.solve(b, x, (2.0 ** f) * a0, omega, prec, tol, maxit, tol_h=tin, tol_s=tin)
            out.append((float(f), solve_bytes(p.npoints, s, sb, db) if st == OK else math.inf, st))
    return out


@dataclass
class AlphaModel:
    """GPR of log2(alpha_best / alpha_ref) against log2(n) for one family,
    precision and omega."""

    gp: GP1D
    prec: int
    omega: float
    data: list
    alpha_ref: object = None

    def predict_log2_factor(self, n: int):
        m, s = self.gp.predict([math.log2(n)])
        return float(m[0]), float(s[0])

    def alpha(self, problem, n: int | None = None) -> float:
        n = n if n is not None else problem.nx
        f, _ = self.predict_log2_factor(n)
        return (2.0 ** f) * self.alpha_ref(problem)


def train(family, sizes, prec: int, omega: float, tol: float, alpha_ref, log2_factors=None, **kw) -> AlphaModel:
    """Sweep alpha on each training size and fit the GP to the best factors.
    alpha_ref(problem): the reference alpha the factors multiply (e.g. the
    closed-form HSS optimum of the family)."""
    log2_factors = log2_factors if log2_factors is not None else np.arange(-4.0, 6.01, 0.5)
    xs, ys, data = [], [], []
    for n in sizes:
        runs = sweep(family, n, prec, omega, log2_factors, tol, alpha_ref, **kw)
        data.append((n, runs))
        ok = [r for r in runs if math.isfinite(r[1])]
        if not ok:
            continue
        f_best = min(ok, key=lambda r: r[1])[0]
        xs.append(math.log2(n))
        ys.append(f_best)
    if not xs:
        raise RuntimeError("no training size converged")
    return AlphaModel(GP1D().fit(xs, ys), prec, omega, data, alpha_ref)
