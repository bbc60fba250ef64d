"""The GP regression behind the data-driven alpha of Sec. 4.2, pinned against
the textbook formulas written out with a dense inverse and SciPy's Gaussian
log-density (CPU only)."""
import math

import numpy as np
import pytest

from paper_2512_21164_gb300 import alpha_gpr as A


def _k(a, b, ell, sf):
    return sf * sf * np.exp(-0.5 * (np.subtract.outer(a, b) / ell) ** 2)


def test_log_marginal_likelihood_equals_gaussian_logpdf():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(3)
    x = np.sort(rng.uniform(0, 5, 7))
    y = np.sin(x) + 0.1 * rng.standard_normal(7)
    for ell, sf, sn in [(0.7, 1.3, 0.2), (2.0, 0.5, 0.05)]:
        cov = _k(x, x, ell, sf) + sn * sn * np.eye(7)
        want = stats.multivariate_normal(mean=np.zeros(7), cov=cov).logpdf(y)
        assert A.log_marginal_likelihood(x, y, ell, sf, sn) == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_posterior_equals_dense_formula():
    """mean = mu + k*^T (K + sn^2 I)^-1 (y - mu), var = k** - k*^T (K + sn^2 I)^-1 k*
    (Rasmussen & Williams eqs. 2.25-2.26) with the hyperparameters fixed."""
    x = np.array([0.0, 1.0, 2.5, 4.0])
    y = np.array([1.0, -0.5, 0.25, 2.0])
    g = A.GP1D().fit(x, y, ells=[1.1], sfs=[0.9], sns=[0.3])
    xs = np.array([-1.0, 0.5, 3.0, 6.0])
    Kinv = np.linalg.inv(_k(x, x, 1.1, 0.9) + 0.09 * np.eye(4))
    ks = _k(xs, x, 1.1, 0.9)
    mu = y.mean()
    mean = mu + ks @ Kinv @ (y - mu)
    var = 0.81 - np.einsum("ij,jk,ik->i", ks, Kinv, ks)
    m, s = g.predict(xs)
    assert np.allclose(m, mean, rtol=1e-12, atol=1e-12)
    assert np.allclose(s, np.sqrt(var), rtol=1e-10, atol=1e-12)


def test_interpolates_with_small_noise_and_uncertainty_grows_away():
    x = np.linspace(0, 6, 9)
    y = np.sin(x)
    g = A.GP1D().fit(x, y, sns=[1e-4])
    m, s = g.predict(x)
    assert np.max(np.abs(m - y)) < 1e-3
    _, s_near = g.predict([3.1])
    _, s_far = g.predict([12.0])
    assert s_far[0] > 10 * s_near[0]


def test_hyperparameters_maximise_the_likelihood_over_the_grid():
    rng = np.random.default_rng(5)
    x = np.linspace(4, 8, 6)
    y = 0.4 * x + 0.05 * rng.standard_normal(6)
    g = A.GP1D().fit(x, y)
    yc = y - y.mean()
    best = A.log_marginal_likelihood(x, yc, g.ell, g.sf, g.sn)
    for ell in (0.5, 1.0, 2.0):
        for sn in (0.05, 0.5):
            assert A.log_marginal_likelihood(x, yc, ell, g.sf, sn) <= best + 1e-12


def test_solve_bytes_is_the_benchmark_byte_model():
    st = dict(outer_its=10, inner_its_h=100, inner_its_s=20)
    # per point: 11 residuals x (3*8 + 2*4) + 120 x 8*4 + 10 x 2*4
    assert A.solve_bytes(1000, st, 4) == 1000 * (11 * 32 + 120 * 32 + 80)
