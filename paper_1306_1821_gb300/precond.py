"""Learned Fourier mass preconditioner for the density HMC move.

The HMC move's diagonal Fourier mass M_k = V_cell/P_k + abar (Eq. Mass_matrix,
kept diagonal in Fourier space as in Sec. 4.1.2) matches the mean precision of
a mode, but inside a survey mask the posterior variance of a large-scale mode
is set mostly by the unobserved volume, where the precision is only the prior
1/lambda_k.  Those directions then oscillate slowly and the chain mixes slowly.
The mass may be any positive operator that does not depend on the density
field (it changes the efficiency, not the target), so a per-bin multiplier s_j
that brings the mass of mass bin j to the measured posterior precision,

    s_j = 1 / (V_j * Mbar_j),   V_j = mean_k Var(delta_k) / N^3,  Mbar_j = mean_k M_k,

(the diagonal "inverse posterior variance" metric of adaptive HMC) is a valid
choice.  A small network learns ln s_j from binned features of a problem: ln P_m
and the binned power ln W_m of the survey window a/abar.  Its training targets
come from plain chains of this library (bps_mass_stats); training runs on the
library's BF16 tensor-core kernels (bps_mlp_*); once installed
(bps_set_mass_net) the library re-evaluates it on the device before every HMC
move from the chain's current P.  This module only arranges those calls.
"""
from dataclasses import dataclass, replace

import numpy as np

from . import bps, inputs

LOG_CLAMP = float(np.log(16.0))
Z_CLAMP = 4.0          # standardised features are clamped to +-4 (as the library does on the device)


@dataclass
class Problem:
    wl: inputs.Workload
    P: np.ndarray        # the power spectrum the statistics are taken at


def random_problems(base, count, seed0, f_sky=(0.2, 0.6), p_scale=(0.5, 2.0), p_jitter=0.1):
    """Surveys like `base` (grid, box, subsamples, radial selection) with a random
    cap (direction and sky fraction) and a random power spectrum: the bin-centre
    spectrum times a random amplitude and a per-bin log-normal jitter."""
    out = []
    for j in range(count):
        rng = np.random.Generator(np.random.PCG64(seed0 + j))
        v = rng.standard_normal(3)
        wl = replace(base, name=f"{base.name}-r{seed0 + j}", f_sky=float(rng.uniform(*f_sky)), seed=seed0 + j,
                     extra={"axis": tuple(v / np.linalg.norm(v))})
        amp = float(np.exp(rng.uniform(np.log(p_scale[0]), np.log(p_scale[1]))))
        P = amp * inputs.bin_centre_spectrum(wl.N, wl.box, wl.n_bins) * np.exp(p_jitter * rng.standard_normal(wl.n_bins))
        out.append(Problem(wl, P))
    return out


def radial_table(wl, n_r=2049):
    """The workload's radial selection sampled at r_j = j (L/2) / (n_r - 1) (inputs recipe)."""
    r = np.arange(n_r) * (wl.box / 2.0 / (n_r - 1))
    if wl.radial == "linear":
        f = np.maximum(0.0, 1.0 - r / (wl.box / 2.0))
    else:
        f = np.exp(-(r / wl.r0) ** 2)
    return np.broadcast_to(f, (wl.n_sub, n_r)).copy()


class DeviceMocks:
    """Surveys of the `inputs` recipe (true field of the workload's spectrum, cap x
    radial response, Poisson counts) made on the device by the library's mock
    calls (bps_mock_*), through one single-chain context of the grid."""

    def __init__(self, wl, stream=None):
        import torch
        self.wl = wl
        N, box = wl.N, wl.box
        self.s = bps.Sampler(N, box, wl.n_sub, wl.n_bins, stream=stream)
        n2 = np.arange(3 * (N // 2) ** 2 + 1, dtype=np.float64)
        self.P = inputs.true_spectrum(2.0 * np.pi * np.sqrt(n2) / box, N, box)
        self.P[0] = 0.0
        self.table = radial_table(wl)
        self.torch = torch

    def make(self, wl, seed):
        """(counts int32, R float32, delta float32) device tensors of one survey."""
        torch = self.torch
        N = wl.N
        d = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
        R = torch.empty((wl.n_sub, N, N, N), dtype=torch.float32, device="cuda")
        c = torch.empty((wl.n_sub, N, N, N), dtype=torch.int32, device="cuda")
        bps.bps_mock_field(self.s.ctx, seed, self.P, d)
        bps.bps_mock_response(self.s.ctx, wl.f_sky, wl.extra.get("axis", (0.0, 0.0, 1.0)), self.table, R)
        bps.bps_mock_counts(self.s.ctx, seed, d, R, wl.b, wl.nbar, 0, c)
        return c, R, d

    def close(self):
        self.s.close()


def features(P, W):
    return np.concatenate([np.log(P), np.log(np.maximum(W, 1e-30))])


def measure(problems, n_mass, n_moves=200, burn_in=100, eps_max=None, n_leapfrog=None, seed=17, stream=None,
            sampler_mass=None, device_mocks=False, chunk=None):
    """Features [count, 2 n_bins] and targets [count, n_mass] from a batch of
    chains (one per problem), with P held at each problem's spectrum.
    Targets: ln s_j = -ln(V_j Mbar_j), clamped to +-ln 16.  V_j is a property of
    the posterior, not of the mass the chains move with: `sampler_mass` (a
    Preconditioner) lets the chains move with a learned mass, whose faster
    mixing gives less biased variances of the slow modes from the same number
    of moves (a second round of training on chains of the improved sampler).
    device_mocks: make the surveys on the device (bps_mock_*) instead of by the
    host recipe; chunk: at most this many chains per batch context."""
    import torch
    if chunk is not None and len(problems) > chunk:
        parts = [measure(problems[i:i + chunk], n_mass, n_moves, burn_in, eps_max, n_leapfrog, seed + i, stream,
                         sampler_mass, device_mocks) for i in range(0, len(problems), chunk)]
        return np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts])
    wl0 = problems[0].wl
    mocks = DeviceMocks(wl0, stream) if device_mocks else None
    cfg = bps.make_config(wl0.n_bins, n_leapfrog=n_leapfrog or wl0.n_leapfrog, eps_max=eps_max or wl0.eps_max,
                          jump=0, fixed_bias_index=0, seed=seed)
    wls = [p.wl for p in problems]
    batch = bps.bps_create_batch([w.N for w in wls], [w.box for w in wls], [w.n_sub for w in wls], cfg, stream)
    try:
        for j, pr in enumerate(problems):
            if mocks is not None:
                c, R, d = mocks.make(pr.wl, pr.wl.seed)
            else:
                delta, counts, Rh = inputs.make_survey(pr.wl)
                c, R = torch.from_numpy(counts).cuda(), torch.from_numpy(Rh).cuda()
                d = torch.from_numpy(delta.astype(np.float32)).cuda()
            bps.bps_batch_set_chain(batch, j, c, R, d, pr.P, np.array(pr.wl.b), np.array(pr.wl.nbar), 0)
            del c, R, d
        n = len(problems)
        W = bps.bps_window_power(batch, wl0.n_bins, n)
        if sampler_mass is not None:
            sampler_mass.install(batch)
        if burn_in:
            bps.bps_mass_stats(batch, burn_in, n_mass, n)
        V, Mb = bps.bps_mass_stats(batch, n_moves, n_mass, n)
        slots = [bps.bps_batch_record_slot(batch, j) for j in range(n)]
    finally:
        bps.bps_destroy(batch)
        if mocks is not None:
            mocks.close()
    feats = np.stack([features(pr.P, W[s]) for pr, s in zip(problems, slots)])
    targ = np.clip(np.stack([-np.log(V[s] * Mb[s]) for s in slots]), -LOG_CLAMP, LOG_CLAMP)
    return feats, targ


def he_init(sizes, seed):
    """Uniform He initialisation (W ~ U(-sqrt(6/n_in), sqrt(6/n_in)), b = 0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = []
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / n_in)
        params.append(rng.uniform(-lim, lim, size=(n_in, n_out)))
        params.append(np.zeros(n_out))
    return params


class Preconditioner:
    """Feature standardisation plus the network (32 -> 128 -> 128 -> n_mass by default)."""

    def __init__(self, n_in, n_mass, hidden=(128, 128), seed=0, stream=None):
        self.sizes = [int(n_in), *[int(h) for h in hidden], int(n_mass)]
        self.net = bps.MLP(self.sizes, stream)
        self.mu = np.zeros(n_in)
        self.sd = np.ones(n_in)
        self.net.set_params(bps.flatten_params(he_init(self.sizes, seed)))

    def fit(self, feats, targ, steps=3000, batch=64, lr=2e-3, seed=1, damping=1.0):
        """Adam on minibatches drawn on the device; returns the last minibatch loss.
        damping (gamma): the network learns gamma * ln s, i.e. M -> s^gamma M.  gamma = 1
        brings each bin's mass to the measured posterior precision (largest gain on the
        slowest bins); smaller gamma stops short of it and costs the fast directions less."""
        import torch
        self.mu = feats.mean(0)
        self.sd = feats.std(0) + 1e-3
        x = torch.from_numpy(self.standardise(feats)).cuda()
        t = torch.from_numpy((damping * targ).astype(np.float32)).cuda()
        return self.net.train(x, t, batch=batch, steps=steps, lr=lr, seed=seed)

    def standardise(self, feats):
        z = (feats.astype(np.float32) - self.mu.astype(np.float32)) / self.sd.astype(np.float32)
        return np.clip(z, -Z_CLAMP, Z_CLAMP).astype(np.float32)

    def predict_log(self, feats):
        import torch
        x = torch.from_numpy(self.standardise(np.atleast_2d(feats))).cuda()
        y = torch.zeros((x.shape[0], self.sizes[-1]), dtype=torch.float32, device="cuda")
        self.net.forward(x, y)
        return np.clip(y.cpu().numpy().astype(np.float64), -LOG_CLAMP, LOG_CLAMP)

    def install(self, ctx):
        """Make the network the per-move mass of a context (single or batch)."""
        bps.bps_set_mass_net(ctx, self.net, self.mu, self.sd, LOG_CLAMP)

    def export(self):
        """The library-format bytes (network, standardisation, clamp) for bps_set_preconditioner."""
        return bps.bps_mlp_export(self.net, self.mu, self.sd, LOG_CLAMP)

    def save(self, path):
        with open(path, "wb") as f:
            f.write(self.export())

    def close(self):
        self.net.close()


def install_saved(ctx, path):
    """Install a preconditioner saved by Preconditioner.save on a context."""
    with open(path, "rb") as f:
        bps.bps_set_preconditioner(ctx, f.read())
