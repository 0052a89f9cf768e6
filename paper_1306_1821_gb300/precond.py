"""Learned Fourier mass preconditioner for the density HMC move.

The HMC move's diagonal Fourier mass M_k = V_cell/P_k + abar (Eq. Mass_matrix,
kept diagonal in Fourier space as in Sec. 4.1.2) balances the prior and the mean
data precision but not the survey geometry: inside a mask most of the posterior
variance of a mode comes from the unobserved volume.  The mass may be any
positive operator that does not depend on the density field (it changes the
efficiency, not the target), so a per-bin multiplier s_j that brings the mass
of mass bin j to the measured posterior precision,

    s_j = 1 / (V_j * Mbar_j),   V_j = mean Var(delta_k)/N^3,  Mbar_j = mean M_k,

is a valid and better-conditioned choice.  A small network learns
log s_j from binned features of a problem (ln P_m and the binned power of the
survey window a/abar), trained on statistics that plain chains of this library
measure (bps_mass_stats); its training and inference kernels are the library's
(bps_mlp_*).  Every step here is a call into the C library; this module only
arranges the calls.
"""
from dataclasses import dataclass

import numpy as np

from . import bps, inputs

LOG_CLAMP = float(np.log(16.0))


@dataclass
class Problem:
    wl: inputs.Workload
    P: np.ndarray        # the power spectrum the statistics are taken at


def random_problems(N, n_bins, count, seed0, n_sub=1, p_scale=(0.5, 2.0), f_sky=(0.2, 0.6)):
    """Surveys with random spectrum amplitude, cap size and cap direction."""
    out = []
    for j in range(count):
        rng = np.random.Generator(np.random.PCG64(seed0 + j))
        v = rng.standard_normal(3)
        wl = inputs.Workload(f"pre{seed0 + j}", N, 500.0 * N / 32.0, n_bins, inputs.SIX_B[:n_sub],
                             [5.0] + inputs._six_nbar()[1:n_sub], float(rng.uniform(*f_sky)), "linear",
                             n_leapfrog=10, eps_max=0.15, seed=seed0 + j, extra={"axis": tuple(v / np.linalg.norm(v))})
        scale = float(np.exp(rng.uniform(np.log(p_scale[0]), np.log(p_scale[1]))))
        P = scale * inputs.bin_centre_spectrum(N, wl.box, n_bins)
        out.append(Problem(wl, P))
    return out


def measure(problems, n_mass, n_moves=200, eps_max=0.15, n_leapfrog=10, seed=17, stream=None):
    """Features [count, 2 n_bins] and targets [count, n_mass] from batched chains.

    Features: ln P_m and ln W_m (window power).  Targets: ln s_j = -ln(V_j Mbar_j),
    clamped to [-ln 16, ln 16]."""
    import torch
    n_bins = problems[0].wl.n_bins
    cfg = bps.make_config(n_bins, n_leapfrog=n_leapfrog, eps_max=eps_max, jump=0, fixed_bias_index=0, seed=seed)
    wls = [p.wl for p in problems]
    batch = bps.bps_create_batch([w.N for w in wls], [w.box for w in wls], [w.n_sub for w in wls], cfg, stream)
    try:
        for j, pr in enumerate(problems):
            delta, counts, R = inputs.make_survey(pr.wl)
            b = np.array(pr.wl.b)
            nbar = np.array(pr.wl.nbar)
            bps.bps_batch_set_chain(batch, j, torch.from_numpy(counts).cuda(), torch.from_numpy(R).cuda(),
                                    torch.from_numpy(delta.astype(np.float32)).cuda(), pr.P, b, nbar, 0)
        W = bps.bps_window_power(batch, n_bins, len(problems))
        V, Mb = bps.bps_mass_stats(batch, n_moves, n_mass, len(problems))
        slots = [bps.bps_batch_record_slot(batch, j) for j in range(len(problems))]
    finally:
        bps.bps_destroy(batch)
    feats = np.stack([np.concatenate([np.log(pr.P), np.log(np.maximum(W[s], 1e-30))])
                      for pr, s in zip(problems, slots)])
    targ = np.clip(np.stack([-np.log(V[s] * Mb[s]) for s in slots]), -LOG_CLAMP, LOG_CLAMP)
    return feats, targ


class Preconditioner:
    """Feature standardisation plus the network; predicts per-mass-bin scales."""

    def __init__(self, n_in, n_mass, hidden=128, seed=0):
        self.sizes = [n_in, hidden, hidden, n_mass]
        self.net = bps.MLP(self.sizes)
        self.mu = np.zeros(n_in)
        self.sd = np.ones(n_in)
        self.net.set_params(bps.flatten_params(he_init(self.sizes, seed)))

    def fit(self, feats, targ, steps=3000, batch=128, lr=2e-3, seed=1):
        import torch
        self.mu = feats.mean(0)
        self.sd = feats.std(0) + 1e-6
        x = torch.from_numpy(((feats - self.mu) / self.sd).astype(np.float32)).cuda()
        t = torch.from_numpy(targ.astype(np.float32)).cuda()
        return self.net.train(x, t, batch=batch, steps=steps, lr=lr, seed=seed)

    def predict_log(self, feats):
        import torch
        x = torch.from_numpy(((np.atleast_2d(feats) - self.mu) / self.sd).astype(np.float32)).cuda()
        y = torch.zeros((x.shape[0], self.sizes[-1]), dtype=torch.float32, device="cuda")
        self.net.forward(x, y)
        return np.clip(y.cpu().numpy().astype(np.float64), -LOG_CLAMP, LOG_CLAMP)

    def scales(self, feats):
        return np.exp(self.predict_log(feats))


def he_init(sizes, seed):
    """Uniform He initialisation (W ~ U(-sqrt(6/n_in), sqrt(6/n_in)), b = 0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = []
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / n_in)
        params.append(rng.uniform(-lim, lim, size=(n_in, n_out)))
        params.append(np.zeros(n_out))
    return params
