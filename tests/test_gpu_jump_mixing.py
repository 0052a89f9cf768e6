"""The deterministic P-delta jump's effect on mixing (Sec. 4.3; the paper's
Conclusion reports correlation lengths of the power spectrum cut by orders of
magnitude).  On the 32^3 survey (one subsample, 40% sky, 16 bins) with the flat
prior on P (alpha = 0, whose posterior is proper for every bin; under the
Jeffreys prior the bins the data barely constrain have an improper marginal at
P -> 0 and no effective sample size to compare), 8000 Gibbs iterations with the
jump on and off: the jump must raise the effective sample size of ln P_m
(Geyer's initial monotone sequence) in the slowest bin and in the median bin
at least threefold, and over the three lowest-k bins by at least half
(geometric mean of the ratios), while the per-bin posterior means of the two chains agree
within five combined Monte Carlo standard errors."""
from dataclasses import replace

import numpy as np
import pytest

from paper_1306_1821_gb300 import diagnostics, inputs

pytestmark = pytest.mark.gpu


def chain(jump, n_iter=8000):
    import torch

    from paper_1306_1821_gb300 import bps
    wl = replace(inputs.WORKLOADS["survey32"], alpha=0.0)
    delta, counts, R = inputs.make_survey(wl)
    P0, b0, nbar0 = inputs.initial_state(wl)
    s = bps.Sampler(wl.N, wl.box, wl.n_sub, wl.n_bins, alpha=0.0, n_leapfrog=wl.n_leapfrog, eps_max=wl.eps_max,
                    jump=int(jump), jump_leapfrog=10, jump_eps_max=0.6, fixed_bias_index=0, seed=3)
    try:
        bps.bps_set_data(s.ctx, torch.from_numpy(counts).cuda(), torch.from_numpy(R).cuda())
        bps.bps_set_state(s.ctx, torch.from_numpy(delta.astype(np.float32)).cuda(), P0, b0, nbar0, 0)
        bps.bps_gibbs_iterate(s.ctx, 300)
        rec = bps.bps_gibbs_iterate(s.ctx, n_iter, s.rec_len)
    finally:
        s.close()
    lnP = np.log(rec[:, :wl.n_bins])
    inside = [m for m in range(wl.n_bins) if (m + 1) * np.sqrt(3.0) * wl.N / 2 / wl.n_bins <= wl.N / 2]
    ess = np.array([diagnostics.ess_geyer(lnP[:, m]) for m in range(wl.n_bins)])
    return lnP, ess, inside


def test_jump_raises_the_effective_sample_size_of_the_power_spectrum():
    lnP_off, ess_off, inside = chain(False)
    lnP_on, ess_on, _ = chain(True)
    print("ESS off", np.round(ess_off[inside], 1))
    print("ESS on ", np.round(ess_on[inside], 1))
    assert ess_on[inside].min() >= 3.0 * ess_off[inside].min()
    assert np.median(ess_on[inside]) >= 3.0 * np.median(ess_off[inside])
    assert np.exp(np.mean(np.log(ess_on[:3] / ess_off[:3]))) >= 1.5
    sd = 0.5 * (lnP_off.std(0) + lnP_on.std(0))
    se = np.sqrt(sd ** 2 / ess_off + sd ** 2 / ess_on)
    assert np.all(np.abs(lnP_on.mean(0) - lnP_off.mean(0))[inside] < 5.0 * se[inside])
