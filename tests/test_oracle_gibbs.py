"""Pins of the oracle's conditional samplers (Secs. 3.4-3.6, 4.2, 4.3, Apps. A-C), the jump with one and two bins."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import gibbs, grid, model
from paper_1306_1821_gb300 import inputs


def survey(N=4, n_sub=2, n_bins=2, seed=2, f_sky=0.8):
    wl = inputs.small_workload(N, n_bins=n_bins, n_sub=n_sub, f_sky=f_sky, seed=seed)
    delta_true, counts, R = inputs.make_survey(wl)
    g = grid.Geometry(N, wl.box, n_bins)
    return wl, g, delta_true, counts, R


def test_bin_power_definition():
    wl, g, d, counts, R = survey(N=8, n_bins=3)
    dh = grid.forward(d)
    s = gibbs.bin_power(g, dh)
    full = np.fft.fftn(d)
    i = np.arange(8)
    n = np.where(i <= 4, i, i - 8)
    n2 = (n[:, None, None] ** 2 + n[None, :, None] ** 2 + n[None, None, :] ** 2)
    b = grid.bin_of_n2(n2, 8, 3)
    for m in range(3):
        assert s[m] == pytest.approx(g.Vc / g.Nv * np.sum(np.abs(full[b == m]) ** 2), rel=1e-12)


def test_power_draw_is_inverse_gamma():
    wl, g, d, counts, R = survey(N=8, n_bins=3)
    dh = grid.forward(d)
    alpha = 1.0
    draws_ = np.array([gibbs.sample_power(g, dh, alpha, 3, it)[0] for it in range(2000)])
    sigma = gibbs.bin_power(g, dh)
    for m in range(3):
        beta = g.n_modes[m] + 2 * alpha - 2
        ref = stats.invgamma(a=beta / 2.0, scale=sigma[m] / 2.0)
        assert stats.kstest(draws_[:, m], ref.cdf).pvalue > 1e-3
    # Eq. INVERSE_GAMMA with a flat prior (alpha = 0) has shape n_m/2 - 1
    d0 = np.array([gibbs.sample_power(g, dh, 0.0, 4, it)[0][2] for it in range(2000)])
    ref0 = stats.invgamma(a=(g.n_modes[2] - 2) / 2.0, scale=sigma[2] / 2.0)
    assert stats.kstest(d0, ref0.cdf).pvalue > 1e-3


def literal_loglik(delta, counts, R, b, nbar, l):
    """log of Eq. LH_per_dataset for subsample l, voxels with R > 0 (normalisation included)."""
    obs = R[l] > 0
    r = R[l][obs].astype(np.float64)
    res = counts[l][obs] - nbar * r * (1.0 + b * delta[obs])
    return -0.5 * np.sum(res * res / (nbar * r)) - 0.5 * obs.sum() * math.log(2 * math.pi * nbar) \
        - 0.5 * np.sum(np.log(r))


def test_bias_conditional_against_quadrature():
    wl, g, d, counts, R = survey(N=4, n_sub=2)
    delta = d * 0.9
    nbar = np.array(wl.nbar)
    sums = gibbs.subsample_sums(delta, counts, R)
    consts = gibbs.data_constants(counts, R)
    l = 1
    # posterior of b_1 by brute-force quadrature of Eq. galaxybias_post (flat prior)
    bs = np.linspace(-6, 8, 4001)
    lp = np.array([literal_loglik(delta, counts, R, bb, nbar[l], l) for bb in bs])
    w = np.exp(lp - lp.max())
    Z = integrate.trapezoid(w, bs)
    mean = integrate.trapezoid(w * bs, bs) / Z
    var = integrate.trapezoid(w * (bs - mean) ** 2, bs) / Z
    xs = np.array([gibbs.sample_bias_norm(delta, sums, consts, wl.b, nbar, 0, 6, it)[0][l] for it in range(3000)])
    assert abs(xs.mean() - mean) < 4 * math.sqrt(var / len(xs))
    assert xs.var() == pytest.approx(var, rel=0.1)
    # fixed index is untouched
    b_new, _ = gibbs.sample_bias_norm(delta, sums, consts, wl.b, nbar, 0, 6, 0)
    assert b_new[0] == wl.b[0]


def test_nbar_conditional_against_quadrature():
    wl, g, d, counts, R = survey(N=4, n_sub=2)
    delta = d * 0.9
    b = np.array(wl.b)
    sums = gibbs.subsample_sums(delta, counts, R)
    consts = gibbs.data_constants(counts, R)
    l = 0
    # Eq. nmean_post with a flat prior: likelihood of Eq. LH_per_dataset in Nbar
    xs_grid = np.linspace(0.5, 25.0, 6001)
    lp = np.array([literal_loglik(delta, counts, R, b[l], x, l) for x in xs_grid])
    w = np.exp(lp - lp.max())
    Z = integrate.trapezoid(w, xs_grid)
    mean = integrate.trapezoid(w * xs_grid, xs_grid) / Z
    var = integrate.trapezoid(w * (xs_grid - mean) ** 2, xs_grid) / Z
    # hold b fixed for the check (fixed index = l), so only Nbar moves
    out = np.array([gibbs.sample_bias_norm(delta, sums, consts, b, wl.nbar, l, 8, it)[1][l] for it in range(3000)])
    assert abs(out.mean() - mean) < 4 * math.sqrt(var / len(out))
    assert out.var() == pytest.approx(var, rel=0.1)


def test_subsample_sums_and_constants():
    wl, g, d, counts, R = survey(N=4, n_sub=2)
    sums = gibbs.subsample_sums(d, counts, R)
    sR, sB, nobs = gibbs.data_constants(counts, R)
    for l in range(2):
        S1 = S2 = S3 = 0.0
        for idx in np.ndindex(4, 4, 4):
            r = float(R[l][idx])
            if r > 0:
                S1 += counts[l][idx] * d[idx]
                S2 += r * d[idx]
                S3 += r * d[idx] ** 2
        assert np.allclose(sums[l], [S1, S2, S3], rtol=1e-12)
        assert nobs[l] == np.sum(R[l] > 0)


@pytest.mark.slow
def test_jump_leaves_conditional_of_P_invariant():
    # 4^3 grid, one bin: theta = ln P is one-dimensional and the whitened field
    # u is invariant under the move, so a chain of jumps must sample
    # p(theta | u, d) ~ exp((1 - alpha) theta) exp(-lik(delta(u, theta)))
    # (Eq. spec_posterior_MIXING_1 with the power-law prior); compare with 1-D quadrature.
    wl, g, d, counts, R = survey(N=4, n_sub=1, n_bins=1, seed=5, f_sky=0.9)
    b = np.array(wl.b)
    nbar = np.array(wl.nbar)
    a, c = model.local_fields(counts, R, b, nbar)
    abar = a.mean()
    alpha = 1.0
    P0 = np.array([inputs.bin_centre_spectrum(4, wl.box, 1)[0]])
    dh0 = grid.forward(d)
    dh0[0, 0, 0] = 0
    ths = np.linspace(math.log(P0[0]) - 8, math.log(P0[0]) + 8, 3001)
    lp = np.array([-gibbs.jump_potential_grad(g, dh0, P0, np.array([t]), a, c, alpha)[0] for t in ths])
    w = np.exp(lp - lp.max())
    Z = integrate.trapezoid(w, ths)
    mean = integrate.trapezoid(w * ths, ths) / Z
    var = integrate.trapezoid(w * (ths - mean) ** 2, ths) / Z
    dh, P = dh0.copy(), P0.copy()
    out = []
    acc = 0
    for it in range(3000):
        dh, P, info = gibbs.jump_move(g, dh, P, a, c, abar, alpha, 6, 0.5, 21, it, P_ref=P0)
        acc += info["accepted"]
        out.append(math.log(P[0]))
    out = np.array(out[200:])
    assert acc > 1500
    nb = 20
    bm = out[: (len(out) // nb) * nb].reshape(nb, -1).mean(1)
    se = bm.std(ddof=1) / math.sqrt(nb)
    assert abs(out.mean() - mean) < 4.5 * max(se, 1e-3)
    assert out.var() == pytest.approx(var, rel=0.15)
    # the whitened field is unchanged by the jumps
    u0 = dh0 / math.sqrt(P0[0])
    assert np.allclose(dh / math.sqrt(P[0]), u0, atol=1e-10)


def test_jump_two_bins_samples_the_conditional_of_P():
    # 4^3 grid, two bins, flat prior alpha = 0 (proper in both tails, so the
    # (alpha - 1) terms of the jump are exercised).  With the whitened field u
    # fixed, delta_hat_k(theta) = delta_hat0_k sqrt(exp(theta_m(k)) / P0_m(k))
    # (Eq. det_trans) and p(theta | u, d) ~ exp((1 - alpha) sum theta -
    # lik(delta(theta))) (Eq. spec_posterior_MIXING_1): written out here with
    # numpy's inverse FFT, apart from the oracle's jump code, on a 2-D grid of
    # (theta_0, theta_1).  A chain of jumps must reproduce its means, variances
    # and correlation.
    wl, g, d, counts, R = survey(N=4, n_sub=1, n_bins=2, seed=5, f_sky=0.9)
    a, c = model.local_fields(counts, R, np.array(wl.b), np.array(wl.nbar))
    abar = a.mean()
    alpha = 0.0
    P0 = inputs.bin_centre_spectrum(4, wl.box, 2)
    lnP0 = np.log(P0)
    dh0 = grid.forward(d)
    dh0[0, 0, 0] = 0
    n = 201
    t0 = np.linspace(lnP0[0] - 9.0, lnP0[0] + 3.0, n)
    t1 = np.linspace(lnP0[1] - 9.0, lnP0[1] + 3.0, n)
    T0, T1 = np.meshgrid(t0, t1, indexing="ij")
    s0 = np.exp(0.5 * (T0 - lnP0[0]))[..., None, None, None]
    s1 = np.exp(0.5 * (T1 - lnP0[1]))[..., None, None, None]
    scale = np.where(g.bin == 0, s0, np.where(g.bin == 1, s1, 0.0))
    delta = np.fft.irfftn(dh0 * scale, s=(4, 4, 4), axes=(-3, -2, -1))
    lik = 0.5 * np.sum(a * delta * delta - 2.0 * c * delta, axis=(-3, -2, -1))
    logp = (1.0 - alpha) * (T0 + T1) - lik
    edge = max(logp[0].max(), logp[-1].max(), logp[:, 0].max(), logp[:, -1].max())
    assert logp.max() - edge > 12.0                     # the grid holds the whole mass
    w = np.exp(logp - logp.max())

    def expect(f):
        return integrate.trapezoid(integrate.trapezoid(w * f, t1, axis=1), t0)

    Z = expect(1.0)
    m = np.array([expect(T0), expect(T1)]) / Z
    v = np.array([expect((T0 - m[0]) ** 2), expect((T1 - m[1]) ** 2)]) / Z
    r = expect((T0 - m[0]) * (T1 - m[1])) / Z / math.sqrt(v[0] * v[1])
    dh, P = dh0.copy(), P0.copy()
    out, acc = [], 0
    for it in range(3200):
        dh, P, info = gibbs.jump_move(g, dh, P, a, c, abar, alpha, 6, 0.5, 21, it, P_ref=P0)
        acc += info["accepted"]
        out.append(np.log(P))
    out = np.array(out[200:])
    assert acc > 2500
    nb = 20
    for k in range(2):
        x = out[:, k]
        bm = x[: (len(x) // nb) * nb].reshape(nb, -1).mean(1)
        se = bm.std(ddof=1) / math.sqrt(nb)
        assert abs(x.mean() - m[k]) < 4.5 * se, (k, x.mean(), m[k], se)
        assert x.var() == pytest.approx(v[k], rel=0.15)
    assert abs(np.corrcoef(out[:, 0], out[:, 1])[0, 1] - r) < 0.1
    # the whitened field is unchanged by the jumps
    lam = np.where(g.bin >= 0, P[np.maximum(g.bin, 0)], 1.0)
    lam0 = np.where(g.bin >= 0, P0[np.maximum(g.bin, 0)], 1.0)
    assert np.allclose(dh / np.sqrt(lam), dh0 / np.sqrt(lam0), atol=1e-10)


def test_jump_gradient_matches_finite_differences():
    wl, g, d, counts, R = survey(N=8, n_sub=2, n_bins=3)
    a, c = model.local_fields(counts, R, np.array(wl.b), np.array(wl.nbar))
    dh0 = grid.forward(d)
    P0 = inputs.bin_centre_spectrum(8, wl.box, 3)
    th = np.log(P0) + np.array([0.2, -0.1, 0.3])
    _, gr = gibbs.jump_potential_grad(g, dh0, P0, th, a, c, 0.5)
    for m in range(3):
        e = np.zeros(3)
        e[m] = 1e-5
        fp = gibbs.jump_potential_grad(g, dh0, P0, th + e, a, c, 0.5)[0]
        fm = gibbs.jump_potential_grad(g, dh0, P0, th - e, a, c, 0.5)[0]
        assert gr[m] == pytest.approx((fp - fm) / 2e-5, rel=1e-6, abs=1e-8)


def test_jump_mass_depends_on_P_only_through_the_whitened_field():
    # the jump moves (delta_hat, P) along delta_hat_k ~ sqrt(P_m(k)) with u fixed
    # (Eq. det_trans); its HMC stays reversible only if the mass is the same at
    # every point of that line, i.e. a function of u (and the fixed P_ref) alone
    wl, g, d, counts, R = survey(N=8, n_sub=1, n_bins=3, seed=4)
    a, _ = model.local_fields(counts, R, np.array(wl.b), np.array(wl.nbar))
    abar = a.mean()
    dh = grid.forward(d)
    P = inputs.bin_centre_spectrum(8, wl.box, 3)
    P_ref = P * np.array([1.3, 0.7, 2.0])
    mu = gibbs.jump_mass(g, dh, P, P_ref, abar)
    assert np.all(mu >= 1.0) and np.any(mu > 1.0)
    rng = np.random.default_rng(8)
    for _ in range(3):
        P2 = P * np.exp(rng.uniform(-2.0, 2.0, 3))
        dh2 = gibbs.jump_field(g, dh, P, np.log(P2))
        assert np.allclose(gibbs.jump_mass(g, dh2, P2, P_ref, abar), mu, rtol=1e-12, atol=0)
