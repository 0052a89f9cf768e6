"""Pins of the oracle's artificial surveys (Sec. 5; App. D; Eq. rel_bias)."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import grid, mock
from paper_1306_1821_gb300 import inputs


def test_exp_neg_matches_the_exponential():
    mu = np.concatenate([np.linspace(0.0, 32.0, 20001), [1e-12, 1e-6, 31.999999]])
    got = mock.exp_neg(mu)
    ref = np.array([math.exp(-x) for x in mu])
    assert np.max(np.abs(got / ref - 1.0)) < 2e-13


@pytest.mark.parametrize("lam", [0.3, 3.0, 17.0, 31.9, 32.1, 100.0, 1000.0])
def test_poisson_counts_follow_the_poisson_law(lam):
    n = 40000
    k = mock.poisson_counts(np.full(n, lam), seed=int(lam * 10) + 1, sub=2)
    assert abs(k.mean() - lam) < 5.0 * math.sqrt(lam / n)
    assert abs(k.var() / lam - 1.0) < 0.05
    # chi-square over the central counts (cells with expected >= 20), tails pooled
    lo, hi = stats.poisson.ppf([1e-4, 1 - 1e-4], lam).astype(int)
    edges = np.arange(lo, hi + 2)
    obs = np.array([np.sum(k < lo)] + [np.sum(k == v) for v in range(lo, hi + 1)] + [np.sum(k > hi)])
    exp = n * np.concatenate([[stats.poisson.cdf(lo - 1, lam)], stats.poisson.pmf(edges[:-1], lam),
                              [stats.poisson.sf(hi, lam)]])
    keep = exp >= 20
    o = np.concatenate([obs[keep], [obs[~keep].sum()]])
    e = np.concatenate([exp[keep], [exp[~keep].sum()]])
    chi2 = np.sum((o - e) ** 2 / np.maximum(e, 1e-300))
    assert stats.chi2.sf(chi2, len(o) - 1) > 1e-3


def test_poisson_counts_zero_mean_and_bounds():
    k = mock.poisson_counts(np.zeros(100), seed=1, sub=0)
    assert np.all(k == 0)
    with pytest.raises(ValueError):
        mock.poisson_counts(np.array([5000.0]), seed=1, sub=0)


def test_gaussian_counts_have_the_papers_noise():
    # N = Nbar R (1 + b delta) + eps, eps ~ N(0, Nbar R), then rounded: mean
    # unchanged and variance Nbar R + 1/12 far from zero
    n = 200000
    delta = np.full(n, 0.3, dtype=np.float32)
    R = np.full(n, 0.8, dtype=np.float32)
    c = mock.gaussian_counts(delta, R, 1.5, 40.0, seed=3, sub=1)
    m = 40.0 * 0.8 * (1 + 1.5 * 0.3)
    assert abs(c.mean() - m) < 5 * math.sqrt(32.0 / n)
    assert abs(c.var() / (32.0 + 1.0 / 12.0) - 1.0) < 0.02
    z = mock.gaussian_counts(np.full(10, -2.0), np.full(10, 1.0), 1.0, 1.0, seed=3, sub=0)
    assert np.all(z >= 0)


def test_mock_field_has_the_prescribed_power():
    N, box = 32, 500.0
    amp = mock.amplitude_table(N, box, lambda k: inputs.true_spectrum(k, N, box))
    d = mock.field(N, amp, seed=5)
    g = grid.Geometry(N, box, 4)
    sel = g.bin >= 0
    ratio = np.abs(grid.forward(d)[sel]) ** 2 / (g.Nv * amp[g.n2[sel]] ** 2)
    w = g.w[sel]
    # E |delta_hat_k|^2 = N_vox A_k^2 for every mode; averaged over the grid
    assert abs(np.sum(w * ratio) / w.sum() - 1.0) < 4.0 / math.sqrt(w.sum())
    assert abs(d.mean()) < 1e-12
    # the field is the inverse transform of A times the transform of the normals
    xi = mock.philox.voxel_normals(5, 0, mock.STAGE_MOCK_FIELD, 0, N ** 3).reshape(N, N, N)
    assert np.allclose(grid.forward(d), amp[g.n2] * grid.forward(xi), atol=1e-9)


def test_schechter_integral_closed_form_matches_quadrature():
    for lo, hi in [(-23.0, -17.0), (-21.4, -21.0), (-18.2, -17.0), (-23.0, -22.6), (-20.0, -20.0)]:
        q = integrate.quad(lambda M: mock.schechter_phi(M), lo, hi, epsabs=0, epsrel=1e-13)[0]
        got = float(mock.schechter_integral(lo, hi))
        assert got == pytest.approx(q, rel=1e-10, abs=1e-300)


def test_comoving_distance_einstein_de_sitter_closed_form():
    # Omega_m = 1: D_C = 2 (c/H0) (1 - 1/sqrt(1+z))
    for z in (0.01, 0.1, 0.5):
        ref = 2.0 * 2997.92458 * (1.0 - 1.0 / math.sqrt(1.0 + z))
        assert mock.comoving_distance(z, 1.0) == pytest.approx(ref, rel=1e-12)
    r = 300.0
    assert mock.comoving_distance(mock.redshift_of(r, 0.24), 0.24) == pytest.approx(r, rel=1e-12)


def test_selection_limits_and_definition():
    M_l, M_u = -21.0, -20.6
    # fully visible where m_bright - mu <= M_l and m_faint - mu >= M_u (r = 150 Mpc/h)
    r = 150.0
    mu = mock.distance_modulus(r, 0.24)
    assert 14.5 - mu <= M_l and 17.77 - mu >= M_u
    assert mock.selection(r, M_l, M_u) == pytest.approx(1.0, rel=1e-12)
    # too bright to be included near the observer
    assert mock.selection(20.0, M_l, M_u) == 0.0
    # invisible beyond the faint limit: mu > m_faint - M_l
    assert mock.selection(5000.0, M_l, M_u) == 0.0
    # partial visibility is the ratio of the integrals of Phi over the visible part
    r = 200.0
    mu = mock.distance_modulus(r, 0.24)
    lo, hi = max(M_l, 14.5 - mu), min(M_u, 17.77 - mu)
    num = integrate.quad(lambda M: mock.schechter_phi(M), lo, hi, epsrel=1e-12)[0]
    den = integrate.quad(lambda M: mock.schechter_phi(M), M_l, M_u, epsrel=1e-12)[0]
    assert mock.selection(r, M_l, M_u) == pytest.approx(num / den, rel=1e-9)


def test_nbar_per_bin_is_additive_and_bias_law_is_anchored():
    edges = np.linspace(-23.0, -17.0, 16)
    nb = mock.nbar_per_bin(edges, phi_star=1.0)
    assert np.sum(nb) == pytest.approx(float(mock.schechter_integral(-23.0, -17.0)), rel=1e-12)
    assert np.all(nb > 0)
    # Eq. rel_bias with a + b = 1: b(M_*) = b_*; brighter galaxies are more biased
    assert float(mock.bias_law(-20.83)) == pytest.approx(1.2, rel=1e-15)
    b = mock.bias_law(0.5 * (edges[:-1] + edges[1:]))
    assert np.all(np.diff(b) < 0)


def test_response_cap_fraction_and_table_interpolation():
    N, box = 64, 500.0
    r_max = box / 2
    table = np.ones((1, 33))
    R = mock.response(N, box, 0.3, (0.2, -0.5, 1.0), table, r_max)[0]
    dx = box / N
    c = (np.arange(N) + 0.5) * dx - box / 2
    x, y, z = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    shell = (r < r_max) & (r > 0.3 * r_max)
    frac = np.sum((R > 0) & shell) / np.sum(shell)
    assert abs(frac - 0.3) < 0.01                      # the cap covers f_sky of the sky
    assert np.all(R[r > r_max] == 0)
    # a table linear in r is reproduced exactly by the interpolation
    lin = np.linspace(1.0, 0.0, 17)[None, :]
    R2 = mock.response(N, box, 1.0, (0, 0, 1), lin, r_max)[0]
    inside = r <= r_max
    assert np.allclose(R2[inside], (1.0 - r / r_max)[inside], atol=1e-6)
