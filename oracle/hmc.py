"""Hybrid Monte Carlo density move of the FP64 oracle (test infrastructure).

Sec. 4.1.1 (Eqs. Potential .. acceptance_rule) and Sec. 4.1.2 (Eqs.
Wiener_Posterior_psi .. Mass_matrix).  The state delta and the momentum p are
real fields; both are held through their half spectra, which is the same
dynamics seen through the transform of App. C.1:
    d delta_hat_k / dt = p_hat_k / M_k          (Eq. HAMILTON1_a, M diagonal in Fourier)
    d p_hat_k / dt     = -grad_hat_k            (Eq. HAMILTON2_a)
Integrator: kick-drift-kick leapfrog (a symplectic scheme, as Sec. 4.1.2
requires).  Trajectory: L_lf steps of size eps = eps_max * u with u uniform in
(0,1), so the pseudo-time tau = L_lf * eps is uniform (Sec. 4.1.2).
Momenta are drawn afresh each move (Sec. 4.1.1): xi ~ N(0, I) on the voxels,
p_hat = sqrt(M_k) FFT(xi), so p ~ N(0, M).
"""
import numpy as np

from . import grid, model, philox


def draw_momentum(geom, M, seed, iteration, sub=0, stage=philox.STAGE_MOMENTUM):
    """p_hat = sqrt(M_k) FFT(xi) with xi the Philox voxel normals of this move."""
    xi = philox.voxel_normals(seed, iteration, stage, sub, geom.Nv).reshape(geom.N, geom.N, geom.N)
    p_hat = np.sqrt(np.where(geom.bin >= 0, M, 0.0)) * grid.forward(xi)
    p_hat[geom.bin < 0] = 0.0
    return p_hat


def move_uniforms(seed, iteration, stage=philox.STAGE_HMC, sub=0):
    """(u_eps, u_accept): the step-size fraction and the MH uniform, both in (0,1)."""
    w = philox.words(seed, iteration, stage, sub, np.zeros(1, dtype=np.uint64))
    u_eps = philox.uniform52(w[0])[0]
    u_acc = philox.uniform52(w[1])[0]
    return u_eps, u_acc


def leapfrog(geom, delta_hat, p_hat, eps, n_steps, P, a, c, invM):
    """Kick-drift-kick leapfrog over n_steps; returns (delta_hat, p_hat, lik_end).

    Kicks use the full force; the first and last kicks are half steps.
    """
    d = delta_hat.copy()
    p = p_hat.copy()
    g, _ = model.gradient_hat(geom, d, P, a, c)
    p -= 0.5 * eps * g
    lik = None
    for s in range(n_steps):
        d += eps * p * invM
        g, lik = model.gradient_hat(geom, d, P, a, c)
        p -= (0.5 * eps if s == n_steps - 1 else eps) * g
    return d, p, lik


def hmc_move(geom, delta_hat, P, a, c, abar, n_steps, eps_max, seed, iteration, mass_scale=None):
    """One HMC move of the density field (Sec. 4.1).

    Returns (new delta_hat, info dict with accepted, dH, eps, H0, H1).
    Accept iff ln(u) < -(H1 - H0)  (Eq. acceptance_rule), FP64 throughout.
    """
    M, invM = model.mass_diag(geom, P, abar, mass_scale)
    p0 = draw_momentum(geom, M, seed, iteration)
    u_eps, u_acc = move_uniforms(seed, iteration)
    eps = eps_max * u_eps
    H0 = model.hamiltonian(geom, delta_hat, p0, P, a, c, invM)
    d1, p1, _ = leapfrog(geom, delta_hat, p0, eps, n_steps, P, a, c, invM)
    H1 = model.hamiltonian(geom, d1, p1, P, a, c, invM)
    dH = H1 - H0
    accepted = bool(np.log(u_acc) < -dH)
    info = dict(accepted=accepted, dH=dH, eps=eps, H0=H0, H1=H1, u_acc=u_acc)
    return (d1 if accepted else delta_hat.copy()), info
