"""Shared set-up of the parity tests: one seeded survey, handed identically to
the CUDA library (through the C ABI) and to the FP64 oracle."""
import numpy as np

from oracle import grid as ogrid
from paper_1306_1821_gb300 import inputs


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def to_f32_spectrum(dh):
    """complex128 half spectrum -> complex64 (the GPU state precision); DC zeroed."""
    out = np.asarray(dh, dtype=np.complex64).copy()
    out[0, 0, 0] = 0
    return out


class Problem:
    """A survey plus a starting state, shared by both sides."""

    def __init__(self, N, n_sub=1, n_bins=4, f_sky=0.6, seed=3, n_leapfrog=5, eps_max=0.3, jump_leapfrog=4,
                 jump_eps_max=0.3, box=None, state_scale=0.8, wl=None, survey=None):
        self.wl = wl or inputs.small_workload(N, box=box, n_bins=n_bins, n_sub=n_sub, f_sky=f_sky, seed=seed,
                                              n_leapfrog=n_leapfrog, eps_max=eps_max,
                                              jump_leapfrog=jump_leapfrog, jump_eps_max=jump_eps_max)
        wl = self.wl
        self.N = wl.N
        # survey: (delta_true, counts, R) made elsewhere (e.g. on the device), else the host recipe
        self.delta_true, self.counts, self.R = survey if survey is not None else inputs.make_survey(wl)
        self.geom = ogrid.Geometry(wl.N, wl.box, wl.n_bins)
        self.P, self.b, self.nbar = inputs.initial_state(wl)
        dh = ogrid.forward(self.delta_true * state_scale)
        self.dh32 = to_f32_spectrum(dh)
        self.dh = self.dh32.astype(np.complex128)

    def config_kwargs(self, seed=11, jump=0):
        wl = self.wl
        return dict(alpha=wl.alpha, n_leapfrog=wl.n_leapfrog, eps_max=wl.eps_max, jump=jump,
                    jump_leapfrog=wl.jump_leapfrog, jump_eps_max=wl.jump_eps_max,
                    fixed_bias_index=wl.fixed_bias, seed=seed)

    def gpu(self, seed=11, iteration=0, jump=0):
        """A library context holding this problem's data and state."""
        import torch

        from paper_1306_1821_gb300 import bps
        s = bps.Sampler(self.N, self.wl.box, self.wl.n_sub, self.wl.n_bins, **self.config_kwargs(seed, jump))
        cnt = torch.from_numpy(self.counts).cuda()
        R = torch.from_numpy(self.R).cuda()
        bps.bps_set_data(s.ctx, cnt, R)
        bps.bps_set_state(s.ctx, None, self.P, self.b, self.nbar, iteration)
        bps.bps_set_spectrum(s.ctx, torch.from_numpy(self.dh32).cuda())
        return s

    def oracle_chain(self, seed=11, iteration=0, jump=False):
        from oracle import gibbs
        wl = self.wl
        return gibbs.Chain(self.geom, self.counts, self.R, self.P, self.b, self.nbar, delta_hat=self.dh,
                           alpha=wl.alpha, n_leapfrog=wl.n_leapfrog, eps_max=wl.eps_max, jump=jump,
                           jump_leapfrog=wl.jump_leapfrog, jump_eps_max=wl.jump_eps_max,
                           fixed_bias=wl.fixed_bias, seed=seed, iteration=iteration)


def gpu_spectrum(s):
    import torch

    from paper_1306_1821_gb300 import bps
    N = s.N
    out = torch.zeros((N, N, N // 2 + 1), dtype=torch.complex64, device="cuda")
    bps.bps_get_spectrum(s.ctx, out)
    return out.cpu().numpy().astype(np.complex128)


def compare_chain(rec, ch, n_iter, tol_dH=1e-3, tol_P=1e-4, tol_b=1e-3, tol_nbar=1e-4, on_iteration=None):
    """Compare GPU chain records rec [n_iter][n_bins + 2 n_sub + 2] with the oracle
    chain `ch` (advanced here), iteration by iteration.

    The two sides take the same Philox draws, so they take the same Metropolis
    decisions unless |dH + ln u| falls inside the FP32 band tol_dH (HMC move and
    jump, Eq. acceptance_rule); after such an iteration the chains are both
    valid but no longer comparable, and the comparison stops.  Returns the
    number of iterations compared and the largest |dH_gpu - dH_oracle|."""
    import math

    from oracle import hmc, philox
    nb, ns = len(ch.P), len(ch.b)
    worst = 0.0
    for i in range(n_iter):
        it = ch.iteration
        r = ch.iterate()
        got = rec[i]
        h = r["hmc"]
        err = abs(got[-2] - h["dH"])
        worst = max(worst, err)
        assert err < tol_dH, (i, got[-2], h["dH"])
        near = abs(h["dH"] + math.log(h["u_acc"])) < tol_dH
        if "jump" in r:
            u_j = hmc.move_uniforms(ch.seed, it, stage=philox.STAGE_JUMP)[1]
            near = near or abs(r["jump"]["dH"] + math.log(u_j)) < tol_dH
        if near:
            return i, worst
        assert int(got[-1]) == int(h["accepted"]), i
        assert np.max(np.abs(got[:nb] / r["P"] - 1)) < tol_P, (i, got[:nb], r["P"])
        assert np.max(np.abs(got[nb:nb + ns] - r["b"])) < tol_b, (i, got[nb:nb + ns], r["b"])
        assert np.max(np.abs(got[nb + ns:nb + 2 * ns] / r["nbar"] - 1)) < tol_nbar, (i,)
        if on_iteration is not None:
            on_iteration(i, r)
    return n_iter, worst
