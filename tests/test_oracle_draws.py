"""Pins of the oracle's scalar samplers against scipy's distributions and
closed-form moments."""
import math

import numpy as np
import pytest
from scipy import special, stats

from oracle import draws, philox


@pytest.mark.parametrize("shape", [0.4, 1.0, 2.5, 40.0, 3.0e4])
def test_gamma_marsaglia_tsang_law(shape):
    n = 3000
    x = np.array([draws.gamma_mt(shape, 5, it, philox.STAGE_POWER, 3)[0] for it in range(n)])
    assert stats.kstest(x, stats.gamma(shape).cdf).pvalue > 1e-3
    assert abs(x.mean() - shape) < 5 * math.sqrt(shape / n)


def test_chi2_two_recipes_agree():
    # Eq. post:posterior_of_x_1 (sum of beta squared normals) and 2 Gamma(beta/2)
    beta = 17
    rng = np.random.default_rng(0)
    a = np.array([draws.chi2_sum_of_squares(beta, rng) for _ in range(3000)])
    b = np.array([2.0 * draws.gamma_mt(beta / 2.0, 1, it, philox.STAGE_POWER, 0)[0] for it in range(3000)])
    assert stats.kstest(a, stats.chi2(beta).cdf).pvalue > 1e-3
    assert stats.kstest(b, stats.chi2(beta).cdf).pvalue > 1e-3
    assert stats.ks_2samp(a, b).pvalue > 1e-3


def test_normal_draw_law():
    z = np.array([draws.normal_draw(9, it, philox.STAGE_BIAS, 2) for it in range(4000)])
    assert stats.kstest(z, "norm").pvalue > 1e-3


def gig_moments(p, A, B):
    """E[x] and Var[x] of GIG(p, A, B) from Bessel-function ratios."""
    w = math.sqrt(A * B)
    eta = math.sqrt(B / A)
    k0 = special.kve(p, w)
    k1 = special.kve(p + 1, w)
    k2 = special.kve(p + 2, w)
    m1 = eta * k1 / k0
    m2 = eta * eta * k2 / k0
    return m1, m2 - m1 * m1


@pytest.mark.parametrize("p,A,B", [(0.5, 2.0, 3.0), (-2.5, 1.0, 4.0), (-0.3, 0.1, 0.2), (3.0, 5.0, 0.5),
                                   (-40.0, 30.0, 800.0)])
def test_gig_small_p_law_and_moments(p, A, B):
    n = 3000
    x = np.array([draws.gig_draw(p, A, B, 4, it, philox.STAGE_NBAR, 1)[0] for it in range(n)])
    ref = stats.geninvgauss(p, math.sqrt(A * B), scale=math.sqrt(B / A))
    assert stats.kstest(x, ref.cdf).pvalue > 1e-3
    m, v = gig_moments(p, A, B)
    assert abs(x.mean() - m) < 5 * math.sqrt(v / n)


def test_gig_large_p_against_normal_limit():
    # |p| ~ 1e6 as in a survey with a million observed voxels.  With x = Nbar,
    # log-density (p-1) ln x - (A x + B/x)/2 is sharply peaked; compare with the
    # Laplace approximation at the mode (its error is O(1/sqrt|p|) in the skewness,
    # far below the tolerance used).
    nobs = 2.0e6
    p = 1.0 - nobs / 2.0
    A = 1.9e6
    B = 4.3e7
    xs = np.array([draws.gig_draw(p, A, B, 8, it, philox.STAGE_NBAR, 0)[0] for it in range(3000)])
    # mode of x^(p-1) exp(-(A x + B/x)/2)
    q = p - 1.0
    mode = (q + math.sqrt(q * q + A * B)) / A
    curv = (p - 1.0) / mode ** 2 + B / mode ** 3           # minus second derivative of log density
    sd = 1.0 / math.sqrt(curv)
    z = (xs - mode) / sd
    assert abs(z.mean()) < 0.1
    assert abs(z.std() - 1.0) < 0.05
    assert stats.kstest(z - z.mean(), "norm").pvalue > 1e-3
    # moments by direct quadrature of the log-density (Bessel functions of order
    # 1e6 overflow in scipy)
    xg = np.linspace(mode - 12 * sd, mode + 12 * sd, 20001)
    lf = (p - 1.0) * np.log(xg / mode) - 0.5 * (A * (xg - mode) + B * (1.0 / xg - 1.0 / mode))
    wq = np.exp(lf)
    Zq = np.trapezoid(wq, xg)
    m = np.trapezoid(wq * xg, xg) / Zq
    v = np.trapezoid(wq * (xg - m) ** 2, xg) / Zq
    assert abs(xs.mean() - m) < 5 * math.sqrt(v / len(xs))
    assert xs.var() == pytest.approx(v, rel=0.1)


def test_gig_bounds_enclose_the_region():
    for lam, omega in [(0.2, 0.5), (1.0, 1.0), (7.0, 3.0), (5.0e5, 2.0e5)]:
        m, vm, vp = draws.gig_bounds(lam, omega)
        ys = m * np.concatenate([np.linspace(1e-3, 0.999, 2000), np.linspace(1.001, 30.0, 4000)])
        vs = (ys - m) * np.exp(0.5 * np.array([draws._gig_logh(y, lam, omega, m) for y in ys]))
        assert vs.max() <= vp * (1 + 1e-9)
        assert vs.min() >= vm * (1 + 1e-9)


@pytest.mark.parametrize("lam,omega", [(2.5, 0.7), (1.0, 3.0), (0.3, 1.5), (-4.0, 0.2), (-2.0e5, 40.0),
                                       (1.0 - 5.0e5, 2.0e3)])
def test_gig_mode_maximises_the_density(lam, omega):
    # h(y) = y^(lam-1) exp(-omega (y + 1/y) / 2): the mode solves
    # (lam - 1) / y - omega (1 - 1/y^2) / 2 = 0 (both branches of the closed form,
    # the second free of cancellation for lam << 0, where the N-bar draw lives)
    m = draws.gig_mode(lam, omega)
    assert m > 0
    dlog = (lam - 1.0) / m - 0.5 * omega * (1.0 - 1.0 / m ** 2)
    assert abs(dlog) <= 1e-10 * (abs(lam - 1.0) / m + omega * (1.0 + 1.0 / m ** 2))
    # brute force: the log density on a fine log-spaced grid around it peaks there
    y = m * np.exp(np.linspace(-0.5, 0.5, 20001))
    logh = (lam - 1.0) * np.log(y) - 0.5 * omega * (y + 1.0 / y)
    assert abs(y[np.argmax(logh)] / m - 1.0) < 1e-4
