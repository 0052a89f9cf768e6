"""Statistical model of the FP64 oracle: prior, data model, potential, forces.

Test infrastructure: imported only by tests, the smoke check and the CPU baseline
of the benchmark.  Every quantity is FP64.

Conventions (readings where the paper is silent):
  * lambda_k = P(|k|) / V_cell is the Fourier-space eigenvalue of the prior
    covariance S of Eq. dens_prior under the App. C.1 convention, so
    (1/2) delta^T S^-1 delta = (1/(2 N_vox)) sum_full |delta_hat_k|^2 / lambda_k.
  * P is piecewise constant on the mode bins (P_m of Sec. 3.4); the DC mode has
    P = 0 (zero-mean field): delta_hat_0 = p_hat_0 = 0 throughout and k = 0
    enters no energy term.
  * the growth factor D+ of Eq. data_model is 1 (dropped in Eq. density_likelihood).
  * every likelihood sum runs over voxels with R > 0 (R = 0 carries no term).
"""
import numpy as np

from . import grid


def local_fields(counts, R, b, nbar):
    """a_i = sum_l b_l^2 Nbar_l R^l_i and c_i = sum_l b_l (N^l_i - Nbar_l R^l_i).

    These are the diagonal curvature and the data drive of the Wiener-posterior
    force, Eq. Wiener_Posterior_force: d psi / d delta = S^-1 delta + a delta - c.
    counts, R: [n_sub, N, N, N]; b, nbar: [n_sub].
    """
    counts = np.asarray(counts, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    a = np.zeros(R.shape[1:])
    c = np.zeros(R.shape[1:])
    for l in range(R.shape[0]):
        obs = R[l] > 0
        a += np.where(obs, b[l] ** 2 * nbar[l] * R[l], 0.0)
        c += np.where(obs, b[l] * (counts[l] - nbar[l] * R[l]), 0.0)
    return a, c


def inv_lambda(geom, P):
    """Per-mode 1/lambda_k = V_cell / P_m (0 on the DC mode)."""
    return geom.per_mode(geom.Vc / np.asarray(P, dtype=np.float64), dc=0.0)


def mass_diag(geom, P, abar, scale=None):
    """Diagonal Fourier mass M_k = 1/lambda_k + abar (Eq. Mass_matrix, Sec. 4.1.2).

    The paper keeps the diagonal of S^-1 + diag(a) in the Fourier basis; the
    Fourier diagonal of diag(a) is its voxel mean abar.  `scale`, if given, is a
    per-mode multiplier (a preconditioner choice; the paper notes the mass
    affects efficiency only, not validity).  Returns (M, 1/M) with 1/M = 0 on DC.
    """
    il = inv_lambda(geom, P)
    M = il + abar
    if scale is not None:
        M = M * scale
    invM = np.where(geom.bin >= 0, 1.0 / np.where(geom.bin >= 0, M, 1.0), 0.0)
    return M, invM


def real_field(geom, delta_hat):
    """delta_i from the half spectrum (Eq. IFFT, C = 1/N_vox)."""
    return grid.inverse(delta_hat, geom.N)


def prior_energy(geom, delta_hat, P):
    """(1/2) delta^T S^-1 delta = (1/(2 N_vox)) sum_k w_k |delta_hat_k|^2 / lambda_k."""
    il = inv_lambda(geom, P)
    return 0.5 / geom.Nv * np.sum(geom.w * np.abs(delta_hat) ** 2 * il)


def likelihood_energy(delta, a, c):
    """(1/2) sum_i (a_i delta_i^2 - 2 c_i delta_i): the delta-dependent part of the
    second term of Eq. Wiener_Posterior_psi (constants dropped)."""
    return 0.5 * np.sum(a * delta * delta - 2.0 * c * delta)


def likelihood_full(delta, counts, R, b, nbar):
    """The second term of Eq. Wiener_Posterior_psi written out literally
    (sum over l and over voxels with R > 0), including the constant."""
    counts = np.asarray(counts, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    tot = 0.0
    for l in range(R.shape[0]):
        obs = R[l] > 0
        res = counts[l][obs] - nbar[l] * R[l][obs] * (1.0 + b[l] * delta[obs])
        tot += 0.5 * np.sum(res * res / (nbar[l] * R[l][obs]))
    return tot


def potential(geom, delta_hat, P, a, c):
    """psi of Eq. Wiener_Posterior_psi up to a delta-independent constant."""
    delta = real_field(geom, delta_hat)
    return prior_energy(geom, delta_hat, P) + likelihood_energy(delta, a, c)


def gradient_hat(geom, delta_hat, P, a, c):
    """Fourier image of the force of Eq. Wiener_Posterior_force.

    grad_i = (S^-1 delta)_i + a_i delta_i - c_i; its forward transform is
    delta_hat_k / lambda_k + FFT(a delta - c)_k.  The DC entry is set to 0
    (the DC mode is frozen at zero by the prior).
    Returns (grad_hat, likelihood_energy at delta).
    """
    delta = real_field(geom, delta_hat)
    g = a * delta - c
    gh = delta_hat * inv_lambda(geom, P) + grid.forward(g)
    gh[geom.bin < 0] = 0.0
    return gh, likelihood_energy(delta, a, c)


def kinetic_energy(geom, p_hat, invM):
    """(1/2) p^T M^-1 p = (1/(2 N_vox)) sum_k w_k |p_hat_k|^2 / M_k (Eq. Hamiltonian)."""
    return 0.5 / geom.Nv * np.sum(geom.w * np.abs(p_hat) ** 2 * invM)


def hamiltonian(geom, delta_hat, p_hat, P, a, c, invM):
    """H = kinetic + psi (Eq. Hamiltonian with the potential of Eq. Wiener_Posterior_psi)."""
    return kinetic_energy(geom, p_hat, invM) + potential(geom, delta_hat, P, a, c)
