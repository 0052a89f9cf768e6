"""Host-side chain analysis: ESS, and the correlation blocks and marginals of
the posterior analysis (Secs. 6.1, 6.2 and 7)."""
import numpy as np

from paper_1306_1821_gb300 import diagnostics


def test_correlation_blocks_of_a_known_covariance():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((7, 7))
    cov = A @ A.T
    corr = diagnostics.correlation(cov)
    sd = np.sqrt(np.diag(cov))
    assert np.allclose(corr, cov / np.outer(sd, sd))
    assert np.allclose(np.diag(corr), 1.0)
    blocks = diagnostics.parameter_blocks(corr, 3, 2)
    assert np.allclose(blocks["b-P"], corr[3:5, 0:3])
    assert np.allclose(blocks["Nbar-P"], corr[5:7, 0:3])
    assert np.allclose(blocks["b-Nbar"], corr[3:5, 5:7])
    # a parameter held fixed (zero variance) has zero correlation, not NaN
    cov[0, :] = cov[:, 0] = 0.0
    assert np.all(np.isfinite(diagnostics.correlation(cov)))


def test_marginal_2d_is_a_density_and_ess_of_white_noise():
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal((2, 20000))
    h, ex, ey = diagnostics.marginal_2d(x, y + 0.5 * x, bins=20)
    assert abs(np.sum(h * np.outer(np.diff(ex), np.diff(ey))) - 1.0) < 1e-12
    ess = diagnostics.ess_geyer(rng.standard_normal(4000))
    assert 3000 < ess < 5500
    # an AR(1) chain with coefficient 0.9 has tau = (1 + 0.9) / (1 - 0.9) = 19
    z = np.empty(40000)
    z[0] = 0.0
    e = rng.standard_normal(40000)
    for i in range(1, z.size):
        z[i] = 0.9 * z[i - 1] + e[i]
    assert abs(z.size / diagnostics.ess_geyer(z) / 19.0 - 1.0) < 0.15


def test_autocorr_against_lag_sums_and_correlation_length_of_ar1():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(257)
    y = x - x.mean()
    v = np.dot(y, y) / x.size
    direct = np.array([np.dot(y[: x.size - n], y[n:]) / x.size / v for n in range(40)])
    assert np.allclose(diagnostics.autocorr(x, 39), direct, rtol=0, atol=1e-12)
    assert np.all(diagnostics.autocorr(np.full(50, 3.0), 5) == 1.0)     # no variance
    # AR(1) with coefficient 0.8: C_n = 0.8^n, below 0.1 first at n = 11
    z = np.empty(200000)
    z[0] = 0.0
    e = rng.standard_normal(z.size)
    for i in range(1, z.size):
        z[i] = 0.8 * z[i - 1] + e[i]
    assert np.allclose(diagnostics.autocorr(z, 12), 0.8 ** np.arange(13), atol=0.02)
    assert diagnostics.correlation_length(z) == 11
