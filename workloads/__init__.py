"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module draws random numbers and lays out problem descriptors; it holds
none of the method's arithmetic (no operator, no residual, no solve).  The
right-hand side b = A x_true is formed by whichever side uses the input: the
oracle in the tests, the library's own FP64 operator in the benchmark.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then two xor-shift-multiply rounds; a uniform double in [0, 1) is the top 53
bits times 2^-53.  Draw order per problem: the scalar parameters (beta, or
kappa then sigma), then x_true by grid index (real part then imaginary part of
each point for complex problems).

The workloads follow the problem classes of Sec. 5 (2D and 3D
convection-diffusion, complex reaction-diffusion) at the grid sizes the
benchmark configurations name; every input is synthetic, there is no dataset.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1

# problem kinds (match the C-ABI and the oracle's numbering)
K_2D5, K_3D7, K_C2D5, K_CSR = 0, 1, 2, 3


class SplitMix64:
    """SplitMix64 generator; `uniform` gives doubles in [0, 1)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_array(self, n: int) -> np.ndarray:
        """n consecutive uniforms, vectorised (same stream as n calls)."""
        if n == 0:
            return np.zeros(0)
        with np.errstate(over="ignore"):
            k = np.arange(1, n + 1, dtype=np.uint64)
            z = np.uint64(self.state) + k * np.uint64(0x9E3779B97F4A7C15)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + n * 0x9E3779B97F4A7C15) & MASK64
        return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class Problem:
    """Descriptor of one linear system (no operator arithmetic here)."""

    kind: int
    nx: int
    ny: int = 1
    nz: int = 1
    h: float = 0.0  # grid spacing; 0 -> 1/(nx+1)
    beta: tuple = (0.0, 0.0, 0.0)
    kappa: float = 0.0
    sigma: float = 0.0
    # CSR (kind K_CSR): host arrays of A, 0-based, int32 / float64
    rowptr: np.ndarray | None = None
    col: np.ndarray | None = None
    val: np.ndarray | None = None
    # complex class: a per-point imaginary diagonal T_i (nx*ny values) instead
    # of sigma I
    sigma_pt: np.ndarray | None = None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def npoints(self) -> int:
        if self.kind == K_CSR:
            return int(len(self.rowptr) - 1)
        return self.nx * self.ny * (self.nz if self.kind == K_3D7 else 1)

    @property
    def nvec(self) -> int:
        """Length of a solution vector in doubles (complex: 2 per point)."""
        return 2 * self.npoints if self.kind == K_C2D5 else self.npoints

    @property
    def hh(self) -> float:
        return self.h if self.h > 0 else 1.0 / (self.nx + 1)


def conv_diff_2d(n: int, seed: int, beta=None, ny: int | None = None) -> tuple[Problem, np.ndarray]:
    """2D convection-diffusion -Lap u + beta.grad u on an n x ny interior grid.

    beta defaults to a draw from U[1,100]^2.  Returns (problem, x_true) with
    x_true ~ U[0,1) by grid index."""
    g = SplitMix64(seed)
    if beta is None:
        beta = (1.0 + 99.0 * g.uniform(), 1.0 + 99.0 * g.uniform())
    ny = n if ny is None else ny
    p = Problem(K_2D5, n, ny, 1, 1.0 / (n + 1), (float(beta[0]), float(beta[1]), 0.0),
                name=f"conv-diff-2d {n}x{ny}")
    return p, g.uniform_array(n * ny)


def conv_diff_3d(n: int, seed: int, bscale=None) -> tuple[Problem, np.ndarray]:
    """3D convection-diffusion on n^3 with beta = (1,1,1) * U[1,50]."""
    g = SplitMix64(seed)
    if bscale is None:
        bscale = 1.0 + 49.0 * g.uniform()
    p = Problem(K_3D7, n, n, n, 1.0 / (n + 1), (bscale, bscale, bscale),
                name=f"conv-diff-3d {n}^3")
    return p, g.uniform_array(n * n * n)


def complex_rd(n: int, seed: int, kappa=None, sigma=None) -> tuple[Problem, np.ndarray]:
    """Complex reaction-diffusion W + iT, W = L + kappa I, T = sigma I, on n x n.

    kappa ~ U[0,10], sigma ~ U[1,100]; x_true interleaved (re, im) ~ U[0,1)."""
    g = SplitMix64(seed)
    if kappa is None:
        kappa = 10.0 * g.uniform()
    if sigma is None:
        sigma = 1.0 + 99.0 * g.uniform()
    p = Problem(K_C2D5, n, n, 1, 1.0 / (n + 1), (0.0, 0.0, 0.0), float(kappa), float(sigma),
                name=f"complex-rd {n}x{n}")
    return p, g.uniform_array(2 * n * n)


def random_csr(n: int, seed: int, extra_per_row: int = 3, skew: float = 0.5) -> tuple[Problem, np.ndarray]:
    """A random sparse nonsymmetric matrix with a positive definite symmetric part.

    Off-diagonal entries: `extra_per_row` random columns per row with values
    U[-1,1); the diagonal is set to (row sum of |off|) * 1.5 + 1 so the
    symmetric part is strictly diagonally dominant (hence positive definite).
    Values are drawn by this module; no operator arithmetic is applied."""
    g = SplitMix64(seed)
    rows = []
    for i in range(n):
        cols = {}
        for _ in range(extra_per_row):
            j = int(g.uniform() * n)
            if j != i:
                cols[j] = (2.0 * g.uniform() - 1.0) * skew
        rows.append(cols)
    offsum = np.zeros(n)
    for i, cols in enumerate(rows):
        for j, v in cols.items():
            offsum[i] += abs(v)
            offsum[j] += abs(v)
    rowptr = [0]
    col, val = [], []
    for i, cols in enumerate(rows):
        cols = dict(cols)
        cols[i] = 1.0 + 1.5 * offsum[i]
        for j in sorted(cols):
            col.append(j)
            val.append(cols[j])
        rowptr.append(len(col))
    p = Problem(K_CSR, n, name=f"random-csr n={n}",
                rowptr=np.asarray(rowptr, np.int32), col=np.asarray(col, np.int32),
                val=np.asarray(val, np.float64))
    return p, g.uniform_array(n)


def paper_cdr_2d(n: int, r: float = 1.0) -> tuple[Problem, np.ndarray]:
    """The 2D convection-diffusion-reaction instance of Sec. 5.2 on n x n:
    A = I (x) T + T (x) I, T = Tridiag(-1, 2, -1) + 2r Tridiag(0.5, 0, -0.5)
    + 100/(n+1)^2 I, r = 1.  With Tridiag(sub, diag, super), T's sub- and
    super-diagonals are -1 + r and -1 - r: in this module's parametrisation
    (W = -1 - c_x, E = -1 + c_x, c = beta h / 2) that is c = -r, i.e.
    beta = -2r/h on both axes.  The reaction enters T_x and T_y, so the
    diagonal is 4 + 200 h^2 (kappa = 200 h^2), as the printed Kronecker sum
    gives.  Sec. 5.2 names no right-hand side; b comes from x = (1, ..., 1)
    as in Sec. 5.3."""
    h = 1.0 / (n + 1)
    p = Problem(K_2D5, n, n, 1, h, (-2.0 * r / h, -2.0 * r / h, 0.0), kappa=200.0 * h * h,
                name=f"paper 2D CDR {n}x{n} (r={r})")
    return p, np.ones(n * n)


def paper_cd_3d(n: int) -> tuple[Problem, np.ndarray]:
    """The 3D convection-diffusion instance of Sec. 5.3 on n^3: T = Tridiag(
    -1 - r, ., -1 + r), r = 1/(2n + 2) = h/2 on every axis, i.e. beta =
    (1, 1, 1); diagonal 6 (the standard 7-point stencil, see the reading on
    the printed diagonal); b from x = (1, ..., 1)."""
    p = Problem(K_3D7, n, n, n, 1.0 / (n + 1), (1.0, 1.0, 1.0), name=f"paper 3D CD {n}^3")
    return p, np.ones(n * n * n)


def paper_complex_rd(n: int, seed: int = 6, s: float = 1e4) -> tuple[Problem, np.ndarray]:
    """The complex reaction-diffusion instance of Sec. 5.4 on n x n:
    -nu Lap w + i V(x) w = f, V = s U[0,1) per grid point (drawn by grid
    index), s = 1e4, nu = 1e-5 (64/n)^2, h = 1/(n+1).  Reading: L is nu times
    the 1/h^2-scaled 5-point Laplacian (the nu ~ 1/n^2 scaling then keeps
    nu/h^2, hence the difficulty, about constant in n).  Multiplying the
    system by h^2/nu gives this module's complex class exactly: M = the
    5-point graph Laplacian (kappa = 0), T_i = (h^2/nu) V_i per point; the
    solution, relative residuals and GADI's iterates (with alpha scaled by
    the same factor) are those of the unscaled system.  b from w = 1 + i at
    every point (Sec. 5.3's recipe; Sec. 5.4 names none)."""
    h = 1.0 / (n + 1)
    nu = 1e-5 * (64.0 / n) ** 2
    g = SplitMix64(seed)
    V = s * g.uniform_array(n * n)
    p = Problem(K_C2D5, n, n, 1, h, (0.0, 0.0, 0.0), 0.0, 0.0, sigma_pt=(h * h / nu) * V,
                name=f"paper complex RD {n}x{n}")
    return p, np.ones(2 * n * n)


def alpha_star(p: Problem) -> float:
    """Closed-form HSS parameter sqrt(lambda_min(M) lambda_max(M)) for the
    stencil classes (Bai, Golub & Ng 2003, cited in Sec. 2.1): the eigenvalues
    of the h^2-scaled graph Laplacian are sums of 4 sin^2(j pi h_/2) terms."""
    def ext(n):
        t = math.pi / (2 * (n + 1))
        return 4 * math.sin(t) ** 2, 4 * math.cos(t) ** 2
    axes = [p.nx, p.ny] + ([p.nz] if p.kind == K_3D7 else [])
    lo = sum(ext(n)[0] for n in axes) + p.kappa
    hi = sum(ext(n)[1] for n in axes) + p.kappa
    return math.sqrt(lo * hi)


# Benchmark / parity configurations (sizes, draws and seeds).
SEED_C1, SEED_C2, SEED_C3, SEED_C4, SEED_C5 = 1, 2, 3, 4, 5


def config1():
    """64 x 64, beta=(10,10), alpha=0.5, omega=1, tol 1e-10, maxit 500, plain FP64."""
    p, xt = conv_diff_2d(64, SEED_C1, beta=(10.0, 10.0))
    return p, xt, dict(alpha=0.5, omega=1.0, tol=1e-10, maxit=500)


def config2(n: int = 2048):
    """2048 x 2048, beta ~ U[1,100]^2 by seed; FP32 inner vs plain FP64."""
    p, xt = conv_diff_2d(n, SEED_C2)
    return p, xt


def config3(n: int = 512):
    """512^3, beta = (1,1,1) U[1,50]; BF16 inner (coefficients BF16)."""
    return conv_diff_3d(n, SEED_C3)


def config4(n: int = 4096):
    """4096 x 4096 complex reaction-diffusion, kappa ~ U[0,10], sigma ~ U[1,100]."""
    return complex_rd(n, SEED_C4)


def config5(nsys: int = 96, nrhs: int = 4, sizes=(128, 256, 512, 1024), seed: int = SEED_C5,
            scaled_alpha: bool = False):
    """Batched: per-system grid N from `sizes`, beta ~ U[1,100]^2,
    alpha ~ logU[1e-2, 10] (or, with scaled_alpha, alpha* of the grid times
    logU[0.5, 2]); nrhs right-hand sides each from x_true ~ U[0,1)."""
    g = SplitMix64(seed)
    systems = []
    for s in range(nsys):
        n = sizes[min(int(g.uniform() * len(sizes)), len(sizes) - 1)]
        beta = (1.0 + 99.0 * g.uniform(), 1.0 + 99.0 * g.uniform())
        if scaled_alpha:
            t = math.pi / (2 * (n + 1))
            a_star = math.sqrt((8 * math.sin(t) ** 2) * (8 * math.cos(t) ** 2))
            alpha = a_star * math.exp(math.log(0.5) + (math.log(2.0) - math.log(0.5)) * g.uniform())
        else:
            alpha = math.exp(math.log(1e-2) + (math.log(10.0) - math.log(1e-2)) * g.uniform())
        p = Problem(K_2D5, n, n, 1, 1.0 / (n + 1), (beta[0], beta[1], 0.0), name=f"sys{s} {n}^2")
        xts = [g.uniform_array(n * n) for _ in range(nrhs)]
        systems.append((p, alpha, xts))
    return systems
