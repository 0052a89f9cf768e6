"""Pins of the oracle's HMC move (Sec. 4.1): reversibility, energy error, and
the Wiener posterior it must sample."""
import numpy as np
import pytest

from oracle import grid, hmc, model, philox
from paper_1306_1821_gb300 import inputs


def setup(N=8, n_sub=1, n_bins=3, seed=11, f_sky=0.6):
    wl = inputs.small_workload(N, n_bins=n_bins, n_sub=n_sub, f_sky=f_sky, seed=seed)
    _, counts, R = inputs.make_survey(wl)
    g = grid.Geometry(N, wl.box, n_bins)
    P = inputs.bin_centre_spectrum(N, wl.box, n_bins)
    a, c = model.local_fields(counts, R, np.array(wl.b), np.array(wl.nbar))
    return g, P, a, c, counts, R, wl


def test_leapfrog_is_reversible():
    g, P, a, c, *_ = setup()
    M, invM = model.mass_diag(g, P, a.mean())
    d0 = inputs.random_spectrum(g.N, g.n_bins, 1, 0.3)
    d0[0, 0, 0] = 0
    p0 = hmc.draw_momentum(g, M, 5, 0)
    d1, p1, _ = hmc.leapfrog(g, d0, p0, 0.2, 15, P, a, c, invM)
    d2, p2, _ = hmc.leapfrog(g, d1, -p1, 0.2, 15, P, a, c, invM)
    assert np.max(np.abs(d2 - d0)) < 1e-12 * np.max(np.abs(d0))
    assert np.max(np.abs(-p2 - p0)) < 1e-12 * np.max(np.abs(p0))


def test_energy_error_is_second_order():
    g, P, a, c, *_ = setup()
    M, invM = model.mass_diag(g, P, a.mean())
    d0 = inputs.random_spectrum(g.N, g.n_bins, 2, 0.3)
    d0[0, 0, 0] = 0
    p0 = hmc.draw_momentum(g, M, 9, 0)
    H0 = model.hamiltonian(g, d0, p0, P, a, c, invM)
    tau = 0.8
    errs = []
    epss = [0.1, 0.05, 0.025, 0.0125]
    for eps in epss:
        n = int(round(tau / eps))
        d1, p1, _ = hmc.leapfrog(g, d0, p0, eps, n, P, a, c, invM)
        errs.append(abs(model.hamiltonian(g, d1, p1, P, a, c, invM) - H0))
    slope = np.polyfit(np.log(epss), np.log(errs), 1)[0]
    assert 1.9 < slope < 2.1


def wiener_dense(g, P, a, c):
    """Mean Q^-1 c and covariance Q^-1 of the Gaussian conditional of delta on the
    zero-mean subspace: Q = S^-1 + diag(a) (Eqs. Wiener_Posterior_psi/force)."""
    N = g.N
    Nv = g.Nv
    # S^-1 on the zero-mean subspace via its Fourier eigenvalues V_cell / P_m
    il = np.zeros(Nv)
    i = np.arange(N)
    s = np.where(i <= N // 2, i, i - N)
    nx, ny, nz = np.meshgrid(s, s, s, indexing="ij")
    b = grid.bin_of_n2((nx ** 2 + ny ** 2 + nz ** 2).ravel(), N, g.n_bins)
    il = np.where(b >= 0, g.Vc / np.asarray(P)[np.maximum(b, 0)], 0.0)
    x = np.stack(np.meshgrid(i, i, i, indexing="ij"), -1).reshape(-1, 3)
    kv = np.stack([nx.ravel(), ny.ravel(), nz.ravel()], -1)
    E = np.exp(2j * np.pi * (x @ kv.T) / N)
    Sinv = ((E * il) @ E.conj().T).real / Nv
    U = np.eye(Nv) - 1.0 / Nv                           # projector off the DC mode
    Q = U @ (Sinv + np.diag(a.ravel())) @ U
    cov = np.linalg.pinv(Q, rcond=1e-12)
    mean = cov @ (U @ c.ravel())
    return mean, cov


@pytest.mark.slow
def test_hmc_samples_the_wiener_posterior():
    g, P, a, c, *_ = setup(N=8, n_bins=3, seed=4, f_sky=0.6)
    mean, cov = wiener_dense(g, P, a, c)
    d = grid.forward(mean.reshape((g.N,) * 3))         # start in the bulk
    n = 3000
    xs = np.empty((n, g.Nv))
    acc = 0
    for it in range(n):
        d, info = hmc.hmc_move(g, d, P, a, c, a.mean(), 8, 0.6, 123, it)
        acc += info["accepted"]
        xs[it] = grid.inverse(d, g.N).ravel()
    assert acc / n > 0.6
    burn = 100
    xs = xs[burn:]
    sd = np.sqrt(np.diag(cov))
    # batch means for the Monte-Carlo error of the mean (accounts for autocorrelation)
    nb = 20
    bm = xs[: (len(xs) // nb) * nb].reshape(nb, -1, g.Nv).mean(1)
    se = bm.std(0, ddof=1) / np.sqrt(nb)
    z = (xs.mean(0) - mean) / se
    assert np.max(np.abs(z)) < 5.5                      # Bonferroni over 512 voxels
    v = xs.var(0)
    assert np.median(np.abs(v / sd ** 2 - 1.0)) < 0.1
    # a few off-diagonal covariances
    emp = np.cov(xs[:, :16].T)
    assert np.max(np.abs(emp - cov[:16, :16])) < 0.15 * np.max(sd[:16] ** 2)


def test_uniform_response_has_closed_form_mode_variance():
    # R == 1 everywhere: Q = S^-1 + abar I is diagonal in Fourier space, so each
    # mode of the Gaussian conditional has variance N_vox / (1/lambda_k + abar)
    # (full-grid |delta_hat_k|^2 normalisation); check the dense route agrees.
    N = 4
    g = grid.Geometry(N, 200.0, 2)
    P = np.array([3.0e5, 1.0e5])
    a = np.full((N, N, N), 2.0)
    c = np.zeros((N, N, N))
    mean, cov = wiener_dense(g, P, a, c)
    assert np.allclose(mean, 0.0, atol=1e-12)
    il = model.inv_lambda(g, P)
    var_hat = np.where(g.bin >= 0, g.Nv / np.where(g.bin >= 0, il + 2.0, 1.0), 0.0)
    # voxel variance from the mode variances: (1/N_vox^2) sum_full var_hat
    vox = np.sum(g.w * var_hat) / g.Nv ** 2
    assert np.allclose(np.diag(cov), vox, rtol=1e-10)


def test_momentum_draw_covariance_is_mass():
    g, P, a, c, *_ = setup(N=4, n_bins=2)
    M, invM = model.mass_diag(g, P, a.mean())
    # E |p_hat_k|^2 = N_vox M_k for every non-DC mode (p ~ N(0, M))
    acc = np.zeros(M.shape)
    n = 4000
    for it in range(n):
        ph = hmc.draw_momentum(g, M, 77, it)
        acc += np.abs(ph) ** 2
    ratio = acc / n / (g.Nv * np.where(g.bin >= 0, M, 1.0))
    r = ratio[g.bin >= 0]
    assert abs(r.mean() - 1.0) < 0.02
    assert np.all(np.abs(r - 1.0) < 0.2)


def test_move_uniforms_follow_counter():
    u1 = hmc.move_uniforms(3, 10)
    u2 = hmc.move_uniforms(3, 11)
    assert u1 != u2 and all(0 < x < 1 for x in u1 + u2)
    w = philox.words(3, 10, philox.STAGE_HMC, 0, np.zeros(1, dtype=np.uint64))
    assert u1[0] == philox.uniform52(w[0])[0]


def test_mass_multipliers_leave_the_closed_form_conditional_unchanged():
    # Sec. 4.1.2: the mass changes only the efficiency of the move, not its
    # target.  With R == 1 the conditional of delta is diagonal in Fourier space:
    # mode k has mean c_hat_k / (1/lambda_k + abar) and full-grid variance
    # N_vox / (1/lambda_k + abar).  HMC moves under strongly non-uniform mass
    # multipliers (a function of |n|^2, so the mass stays that of a real field)
    # must reproduce both.
    N = 4
    g = grid.Geometry(N, 200.0, 2)
    P = np.array([3.0e5, 1.0e5])
    abar = 2.0
    a = np.full((N, N, N), abar)
    rng = np.random.Generator(np.random.PCG64(17))
    c = rng.standard_normal((N, N, N))
    il = model.inv_lambda(g, P)
    q = np.where(g.bin >= 0, il + abar, 1.0)
    mean_hat = np.where(g.bin >= 0, grid.forward(c) / q, 0.0)
    var_hat = np.where(g.bin >= 0, g.Nv / q, 0.0)
    levels = np.unique(g.n2)
    per_level = dict(zip(levels.tolist(), np.exp(rng.uniform(np.log(1 / 8), np.log(8), len(levels)))))
    scale = np.vectorize(per_level.get)(g.n2).astype(np.float64)
    d = mean_hat.copy()
    n, acc = 6000, 0
    s1 = np.zeros(d.shape, dtype=np.complex128)
    s2 = np.zeros(d.shape)
    for it in range(n):
        d, info = hmc.hmc_move(g, d, P, a, c, abar, 6, 0.9, 29, it, mass_scale=scale)
        acc += info["accepted"]
        s1 += d
        s2 += np.abs(d - mean_hat) ** 2
    assert acc / n > 0.6
    obs = g.bin >= 0
    # mean: per-mode z-scores against the closed form (moves are close to
    # independent at this size; allow 4.5 sigma over the modes)
    z = np.abs(s1 / n - mean_hat)[obs] / np.sqrt(var_hat[obs] / n)
    assert np.max(z) < 4.5 * np.sqrt(3.0)
    # variance: the mean ratio over all modes and over each mass level
    r = (s2 / n)[obs] / var_hat[obs]
    assert abs(r.mean() - 1.0) < 0.03
    for lev in levels[levels > 0]:
        sel = (g.n2 == lev)[obs]
        assert abs(r[sel].mean() - 1.0) < 0.15, (lev, r[sel].mean())


def test_leapfrog_energy_error_telescopes_for_quadratic_potential():
    # The potential of the density move is exactly quadratic in delta (Eq.
    # Wiener_Posterior_psi at fixed P, b, Nbar), and for kick-drift-kick
    # leapfrog on a quadratic potential each step changes H by
    # (eps^2/8)(g_{n+1}^T M^-1 g_{n+1} - g_n^T M^-1 g_n), so the energy error of
    # a whole trajectory is (eps^2/8)(g_L^T M^-1 g_L - g_0^T M^-1 g_0).  The CUDA
    # library evaluates Delta H of Eq. acceptance_rule this way; here the
    # identity is checked against the direct difference H1 - H0 of the oracle,
    # with and without mass multipliers.
    g, P, a, c, *_ = setup(N=16, n_sub=2, n_bins=4, seed=3)
    d0 = inputs.random_spectrum(g.N, g.n_bins, 1, 0.3)
    d0[0, 0, 0] = 0

    def gnorm(d, invM):
        gh, _ = model.gradient_hat(g, d, P, a, c)
        return np.sum(g.w * np.abs(gh) ** 2 * invM) / g.Nv

    levels = np.unique(g.n2)
    per_level = dict(zip(levels.tolist(), np.exp(np.random.default_rng(2).uniform(-1, 1, len(levels)))))
    for scale in (None, np.vectorize(per_level.get)(g.n2).astype(np.float64)):
        M, invM = model.mass_diag(g, P, a.mean(), scale)
        p0 = hmc.draw_momentum(g, M, 5, 0)
        H0 = model.hamiltonian(g, d0, p0, P, a, c, invM)
        for eps, L in [(0.05, 3), (0.1, 7), (0.3, 20)]:
            d1, p1, _ = hmc.leapfrog(g, d0, p0, eps, L, P, a, c, invM)
            dH = model.hamiltonian(g, d1, p1, P, a, c, invM) - H0
            ident = eps ** 2 / 8.0 * (gnorm(d1, invM) - gnorm(d0, invM))
            assert abs(dH) > 1e-2
            assert abs(dH - ident) < 1e-10 * max(1.0, abs(dH))
