"""Pins of the oracle's model: prior, likelihood, potential, force, mass."""
import numpy as np
import pytest

from oracle import grid, model
from paper_1306_1821_gb300 import inputs


def dense_S(geom, P):
    """Prior covariance S as an explicit N_vox x N_vox matrix built from the
    definition 'Fourier transform of S is the power spectrum' (Sec. 3.3.1):
    S_ij = (1/N_vox) sum_k lambda_k exp(i k (x_i - x_j)), lambda_k = P_k / V_cell."""
    N = geom.N
    i = np.arange(N)
    s = np.where(i <= N // 2, i, i - N)
    nx, ny, nz = np.meshgrid(s, s, s, indexing="ij")
    n2 = (nx ** 2 + ny ** 2 + nz ** 2).ravel()
    b = grid.bin_of_n2(n2, N, geom.n_bins)
    lam = np.where(b >= 0, np.asarray(P)[np.maximum(b, 0)] / geom.Vc, 0.0)
    x = np.stack(np.meshgrid(i, i, i, indexing="ij"), -1).reshape(-1, 3)
    kvec = np.stack([nx.ravel(), ny.ravel(), nz.ravel()], -1)
    E = np.exp(2j * np.pi * (x @ kvec.T) / N)            # [voxel, mode]
    S = (E * lam) @ E.conj().T / N ** 3
    return S.real, E


def small_problem(N=4, n_sub=2, seed=3, n_bins=2):
    wl = inputs.small_workload(N, n_bins=n_bins, n_sub=n_sub, f_sky=0.7, seed=seed)
    _, counts, R = inputs.make_survey(wl)
    g = grid.Geometry(N, wl.box, n_bins)
    P = inputs.bin_centre_spectrum(N, wl.box, n_bins)
    return wl, g, counts, R, P


def test_prior_energy_equals_dense_quadratic_form():
    wl, g, counts, R, P = small_problem()
    S, E = dense_S(g, P)
    rng = np.random.default_rng(0)
    d = rng.standard_normal(g.Nv)
    d -= d.mean()                                      # DC frozen at zero
    dh = grid.forward(d.reshape(g.N, g.N, g.N))
    # S is singular only on the constant vector; the pseudo-inverse is the
    # inverse on the zero-mean subspace
    dense = 0.5 * d @ np.linalg.pinv(S, rcond=1e-12) @ d
    assert model.prior_energy(g, dh, P) == pytest.approx(dense, rel=1e-10)


def test_likelihood_energy_is_literal_likelihood_up_to_constant():
    wl, g, counts, R, P = small_problem()
    b = np.array([1.3, 0.8])
    nbar = np.array([4.0, 2.5])
    a, c = model.local_fields(counts, R, b, nbar)
    rng = np.random.default_rng(1)
    diffs = []
    for _ in range(4):
        d = 0.3 * rng.standard_normal((g.N,) * 3)
        diffs.append(model.likelihood_full(d, counts, R, b, nbar) - model.likelihood_energy(d, a, c))
    assert np.ptp(diffs) < 1e-10 * max(1.0, abs(diffs[0]))


def test_gradient_matches_finite_differences():
    wl, g, counts, R, P = small_problem(N=8, n_sub=2, n_bins=3)
    b = np.array([1.1, 1.6])
    nbar = np.array([3.0, 1.5])
    a, c = model.local_fields(counts, R, b, nbar)
    rng = np.random.default_rng(2)
    d = 0.4 * rng.standard_normal((g.N,) * 3)
    d -= d.mean()
    dh = grid.forward(d)
    gh, lik = model.gradient_hat(g, dh, P, a, c)
    G = grid.inverse(gh, g.N)                           # real-space force d psi / d delta_i
    assert lik == pytest.approx(model.likelihood_energy(d, a, c), rel=1e-12)
    for t in range(4):
        v = rng.standard_normal((g.N,) * 3)
        v -= v.mean()
        vh = grid.forward(v)
        h = 1e-4
        fd = (model.potential(g, dh + h * vh, P, a, c) - model.potential(g, dh - h * vh, P, a, c)) / (2 * h)
        assert np.sum(G * v) == pytest.approx(fd, rel=1e-7)


def test_force_is_dense_precision_times_delta_minus_drive():
    # Eq. Wiener_Posterior_force written with dense matrices at 4^3
    wl, g, counts, R, P = small_problem()
    b = np.array([1.2, 1.0])
    nbar = np.array([5.0, 2.0])
    a, c = model.local_fields(counts, R, b, nbar)
    S, _ = dense_S(g, P)
    rng = np.random.default_rng(5)
    d = rng.standard_normal(g.Nv)
    d -= d.mean()
    force = np.linalg.pinv(S, rcond=1e-12) @ d + a.ravel() * d - c.ravel()
    gh, _ = model.gradient_hat(g, grid.forward(d.reshape((g.N,) * 3)), P, a, c)
    G = grid.inverse(gh, g.N).ravel()
    # the oracle force has its DC component removed (DC frozen); compare zero-mean parts
    assert np.allclose(G, force - force.mean(), atol=1e-9)


def test_mass_and_kinetic_energy_dense():
    wl, g, counts, R, P = small_problem()
    abar = 0.7
    M, invM = model.mass_diag(g, P, abar)
    # M as an operator: Fourier eigenvalues M_k = 1/lambda_k + abar (Eq. Mass_matrix, Fourier diagonal)
    S, _ = dense_S(g, P)
    Sinv = np.linalg.pinv(S, rcond=1e-12)
    proj = np.eye(g.Nv) - np.full((g.Nv, g.Nv), 1.0 / g.Nv)
    Mop = Sinv + abar * proj
    rng = np.random.default_rng(6)
    p = rng.standard_normal(g.Nv)
    p -= p.mean()
    ph = grid.forward(p.reshape((g.N,) * 3))
    dense = 0.5 * p @ np.linalg.pinv(Mop, rcond=1e-12) @ p
    assert model.kinetic_energy(g, ph, invM) == pytest.approx(dense, rel=1e-10)
    assert invM[0, 0, 0] == 0.0
