"""Conditional samplers and the multiple-block scan of the FP64 oracle.

Test infrastructure: imported only by tests, the smoke check and the CPU
baseline of the benchmark.

Scan order (Sec. 3.2, Eq. multiblock; Fig. 1): the paper lists delta, S, Nbar, b
in the equation and delta, b, P, Nbar in the flow chart.  Any fixed order that
conditions on the latest values is a valid Gibbs scan; this oracle (and the
CUDA library) uses
    delta (HMC, Sec. 4.1) -> P (Sec. 4.2) -> [P-delta jump, Sec. 4.3/App. C]
    -> b (Sec. 3.5) -> Nbar (Sec. 3.6) -> rebuild of the local fields a, c.

Readings where the paper is silent or inconsistent:
  * sigma_m = (V_cell / N_vox) sum_{k in m} w_k |delta_hat_k|^2 (full-grid sum)
    and n_m = the full-grid mode count, which makes Eq. INVERSE_GAMMA the exact
    conditional of P_m under the prior of Eq. dens_prior.
  * bias conditional (Sec. 3.5, App. B): the variance is 1/C with
    C = Nbar sum R delta^2 and the mean D/C with D = sum (N - Nbar R) delta (the
    forms the App. B expansion gives; the printed 1/sum Nbar R delta and
    sum (N - Nbar) delta are typos).  Sums over R > 0.
  * GIG shape p = 1 - N_obs/2 with N_obs the number of voxels with R > 0
    (Sec. 3.6; App. A's 1 - N_vox/2 counts unobserved voxels, which carry no
    likelihood term).
  * one bias (index `fixed_bias`) is held fixed: b and P are exactly
    degenerate (delta -> delta/k, b -> k b, P -> P/k^2), and the paper fixes
    one luminosity bin's bias (Secs. 6.2 and 7).
  * the jump (Sec. 4.3, App. C, Eq. spec_posterior_MIXING_1): with the whitened
    field u_k = delta_hat_k / sqrt(lambda_k) held fixed, P is updated from
    p(P | u, d) ~ prior(P) x likelihood(delta(u, P)) and then
    delta_hat_k <- sqrt(P'_m / P_m) delta_hat_k (Eq. det_trans).  The update of P
    is an HMC in theta_m = ln P_m (the paper uses an HMC there): potential
    psi_J = sum_m (alpha - 1) theta_m + (1/2) sum_i (a delta^2 - 2 c delta).
    Its diagonal mass must not depend on P (the variable the move updates), or
    the move would not be reversible; it is built from the whitened field u,
    abar and a reference spectrum P_ref held fixed between state resets:
        mu_m = max(1, (abar / (4 N_vox)) (P_ref_m / V_cell) sum_{k in m} w_k |u_k|^2)
             = max(1, abar P_ref_m sigma_m / (4 V_cell P_m)),
    the curvature of the likelihood term in theta_m at P = P_ref.
"""
import math

import numpy as np

from . import draws, grid, hmc, model, philox


def bin_power(geom, delta_hat):
    """sigma_m of Sec. 3.4 with the normalisation stated above (FP64)."""
    e = geom.w * np.abs(delta_hat) ** 2
    s = np.bincount(geom.bin[geom.bin >= 0], weights=e[geom.bin >= 0], minlength=geom.n_bins)
    return s * geom.Vc / geom.Nv


def sample_power(geom, delta_hat, alpha, seed, iteration):
    """P_m = sigma_m / x_m, x_m ~ chi^2_{beta_m}, beta_m = n_m + 2 alpha - 2 (Sec. 4.2)."""
    sigma = bin_power(geom, delta_hat)
    beta = geom.n_modes + 2.0 * alpha - 2.0
    P = np.empty(geom.n_bins)
    for m in range(geom.n_bins):
        g, _ = draws.gamma_mt(0.5 * beta[m], seed, iteration, philox.STAGE_POWER, m)
        P[m] = sigma[m] / (2.0 * g)
    return P, sigma


def data_constants(counts, R):
    """Per-subsample constants fixed by the data: (sum R, sum N^2/R, N_obs), over R > 0."""
    counts = np.asarray(counts, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    n_sub = R.shape[0]
    sR = np.zeros(n_sub)
    sB = np.zeros(n_sub)
    nobs = np.zeros(n_sub)
    for l in range(n_sub):
        obs = R[l] > 0
        sR[l] = R[l][obs].sum()
        sB[l] = (counts[l][obs] ** 2 / R[l][obs]).sum()
        nobs[l] = obs.sum()
    return sR, sB, nobs


def subsample_sums(delta, counts, R):
    """S1 = sum N delta, S2 = sum R delta, S3 = sum R delta^2 per subsample (R > 0)."""
    counts = np.asarray(counts, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    out = np.zeros((R.shape[0], 3))
    for l in range(R.shape[0]):
        obs = R[l] > 0
        d = delta[obs]
        out[l, 0] = np.sum(counts[l][obs] * d)
        out[l, 1] = np.sum(R[l][obs] * d)
        out[l, 2] = np.sum(R[l][obs] * d * d)
    return out


def sample_bias_norm(delta, sums, consts, b, nbar, fixed_bias, seed, iteration):
    """b_l ~ N(D/C, 1/C) (Sec. 3.5, App. B) then Nbar_l ~ GIG(p, A, B) (Sec. 3.6, App. A)."""
    sR, sB, nobs = consts
    b = np.array(b, dtype=np.float64)
    nbar = np.array(nbar, dtype=np.float64)
    for l in range(len(b)):
        S1, S2, S3 = sums[l]
        if l != fixed_bias:
            C = nbar[l] * S3
            D = S1 - nbar[l] * S2
            z = draws.normal_draw(seed, iteration, philox.STAGE_BIAS, l)
            b[l] = D / C + z / math.sqrt(C)
        A = sR[l] + 2.0 * b[l] * S2 + b[l] * b[l] * S3
        p = 1.0 - 0.5 * nobs[l]
        nbar[l], _ = draws.gig_draw(p, A, sB[l], seed, iteration, philox.STAGE_NBAR, l)
    return b, nbar


def jump_mass(geom, delta_hat, P, P_ref, abar):
    """mu_m = max(1, abar P_ref_m sigma_m / (4 V_cell P_m)); depends on P only through u."""
    sigma = bin_power(geom, delta_hat)
    return np.maximum(1.0, abar * np.asarray(P_ref) * sigma / (4.0 * geom.Vc * np.asarray(P)))


def jump_field(geom, delta_hat0, P0, theta):
    """delta_hat(theta)_k = sqrt(exp(theta_m) / P0_m) delta_hat0_k (Eq. det_trans)."""
    r = np.sqrt(np.exp(theta) / P0)
    return delta_hat0 * geom.per_mode(r, dc=0.0)


def jump_potential_grad(geom, delta_hat0, P0, theta, a, c, alpha):
    """psi_J(theta) and d psi_J / d theta_m (see module docstring)."""
    dh = jump_field(geom, delta_hat0, P0, theta)
    delta = grid.inverse(dh, geom.N)
    lik = model.likelihood_energy(delta, a, c)
    gh = grid.forward(a * delta - c)
    e = geom.w * np.real(np.conj(gh) * dh)
    s = np.bincount(geom.bin[geom.bin >= 0], weights=e[geom.bin >= 0], minlength=geom.n_bins)
    grad = (alpha - 1.0) + 0.5 / geom.Nv * s
    psi = (alpha - 1.0) * np.sum(theta) + lik
    return psi, grad


def jump_move(geom, delta_hat, P, a, c, abar, alpha, n_steps, eps_max, seed, iteration, P_ref=None):
    """Deterministic P-delta transition with an HMC in theta = ln P (Sec. 4.3, App. C)."""
    mu = jump_mass(geom, delta_hat, P, P if P_ref is None else P_ref, abar)
    rho0 = np.array([draws.normal_draw(seed, iteration, philox.STAGE_JUMP_MOM, m) for m in range(geom.n_bins)])
    rho0 = rho0 * np.sqrt(mu)
    u_eps, u_acc = hmc.move_uniforms(seed, iteration, stage=philox.STAGE_JUMP)
    eps = eps_max * u_eps
    th0 = np.log(P)
    psi0, g = jump_potential_grad(geom, delta_hat, P, th0, a, c, alpha)
    H0 = 0.5 * np.sum(rho0 ** 2 / mu) + psi0
    th = th0.copy()
    rho = rho0 - 0.5 * eps * g
    psi = psi0
    for s in range(n_steps):
        th = th + eps * rho / mu
        psi, g = jump_potential_grad(geom, delta_hat, P, th, a, c, alpha)
        rho = rho - (0.5 * eps if s == n_steps - 1 else eps) * g
    H1 = 0.5 * np.sum(rho ** 2 / mu) + psi
    dH = H1 - H0
    accepted = bool(np.log(u_acc) < -dH)
    info = dict(accepted=accepted, dH=dH, eps=eps, H0=H0, H1=H1)
    if accepted:
        return jump_field(geom, delta_hat, P, th), np.exp(th), info
    return delta_hat.copy(), np.array(P, dtype=np.float64), info


class Chain:
    """Oracle state of one chain: delta_hat, P, b, Nbar and the iteration counter."""

    def __init__(self, geom, counts, R, P, b, nbar, delta_hat=None, alpha=1.0, n_leapfrog=10,
                 eps_max=0.3, jump=False, jump_leapfrog=10, jump_eps_max=0.1, fixed_bias=0,
                 seed=0, iteration=0):
        self.geom = geom
        self.counts = np.asarray(counts)
        self.R = np.asarray(R, dtype=np.float64)
        self.P = np.array(P, dtype=np.float64)
        self.b = np.array(b, dtype=np.float64)
        self.nbar = np.array(nbar, dtype=np.float64)
        N = geom.N
        self.delta_hat = (np.zeros((N, N, N // 2 + 1), dtype=np.complex128)
                          if delta_hat is None else np.array(delta_hat, dtype=np.complex128))
        self.alpha = alpha
        self.n_leapfrog = n_leapfrog
        self.eps_max = eps_max
        self.jump = jump
        self.jump_leapfrog = jump_leapfrog
        self.jump_eps_max = jump_eps_max
        self.fixed_bias = fixed_bias
        self.seed = seed
        self.iteration = iteration
        self.P_ref = self.P.copy()
        self.mass_fn = None
        self.consts = data_constants(self.counts, self.R)
        self.rebuild()

    def rebuild(self):
        self.a, self.c = model.local_fields(self.counts, self.R, self.b, self.nbar)
        self.abar = float(np.mean(self.a))

    def hmc_step(self):
        # mass_fn (optional): chain -> per-mode multipliers of the diagonal mass,
        # a function of the hyperparameters only (Sec. 4.1.2 leaves the mass free)
        scale = self.mass_fn(self) if self.mass_fn is not None else None
        self.delta_hat, info = hmc.hmc_move(self.geom, self.delta_hat, self.P, self.a, self.c, self.abar,
                                            self.n_leapfrog, self.eps_max, self.seed, self.iteration, scale)
        return info

    def sample_power(self):
        self.P, sigma = sample_power(self.geom, self.delta_hat, self.alpha, self.seed, self.iteration)
        return sigma

    def jump_step(self):
        self.delta_hat, self.P, info = jump_move(self.geom, self.delta_hat, self.P, self.a, self.c, self.abar,
                                                 self.alpha, self.jump_leapfrog, self.jump_eps_max,
                                                 self.seed, self.iteration, self.P_ref)
        return info

    def sample_bias_norm(self):
        delta = grid.inverse(self.delta_hat, self.geom.N)
        sums = subsample_sums(delta, self.counts, self.R)
        self.b, self.nbar = sample_bias_norm(delta, sums, self.consts, self.b, self.nbar,
                                             self.fixed_bias, self.seed, self.iteration)
        self.rebuild()
        return sums

    def iterate(self):
        """One full Gibbs iteration in the scan order of the module docstring."""
        rec = {}
        rec["hmc"] = self.hmc_step()
        self.sample_power()
        if self.jump:
            rec["jump"] = self.jump_step()
        self.sample_bias_norm()
        rec["P"] = self.P.copy()
        rec["b"] = self.b.copy()
        rec["nbar"] = self.nbar.copy()
        self.iteration += 1
        return rec
