"""What the trained network mass gains over the plain diagonal mass.

The network is trained on the device (BF16 kernels) on statistics of plain
chains of 32^3 surveys with random caps and spectra, then installed on a
held-out survey (the 32^3 survey of the benchmark set: 40% sky, linear radial
fall-off, one subsample).  At fixed P, an HMC chain of the density field is run
with the plain mass and with the network mass, same seed and step size; the
statistic is ln sigma_m, the k-bin power of delta (the quantity the power
spectrum draw conditions on).

Checks: (1) on held-out training-style problems the network predicts the
measured log multipliers better than the plain mass does (ln s = 0);
(2) the effective sample size of the slowest bins, and the minimum over all
bins, is several times larger with the network mass; (3) both chains sample
the same distribution: the per-bin means of ln sigma_m agree within five
combined Monte Carlo standard errors (sd / sqrt(ESS))."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N_MASS = 16
N_MOVES = 3000


@pytest.fixture(scope="module")
def trained():
    from paper_1306_1821_gb300 import inputs, precond
    probs = precond.random_problems(inputs.WORKLOADS["survey32"], 160, 7000, p_jitter=0.3)
    F, T = precond.measure(probs, N_MASS, n_moves=300, burn_in=100)
    pc = precond.Preconditioner(F.shape[1], N_MASS)
    pc.fit(F[:-16], T[:-16], steps=2000, batch=64)
    yield pc, F[-16:], T[-16:]
    pc.close()


def chain_stats(pc, eps, seed):
    import torch

    from paper_1306_1821_gb300 import bps, diagnostics, inputs
    wl = inputs.WORKLOADS["survey32"]
    N = wl.N
    delta, counts, R = inputs.make_survey(wl)
    P0, b0, n0 = inputs.initial_state(wl)
    s = bps.Sampler(N, wl.box, wl.n_sub, wl.n_bins, n_leapfrog=10, eps_max=eps, jump=0, fixed_bias_index=0,
                    seed=seed)
    try:
        bps.bps_set_data(s.ctx, torch.from_numpy(counts).cuda(), torch.from_numpy(R).cuda())
        bps.bps_set_state(s.ctx, torch.from_numpy(delta.astype(np.float32)).cuda(), P0, b0, n0, 0)
        if pc is not None:
            pc.install(s.ctx)
        for _ in range(200):
            bps.bps_hmc_step(s.ctx, False)
        spec = torch.zeros((N, N, N // 2 + 1), dtype=torch.complex64, device="cuda")
        sig = torch.zeros(wl.n_bins, dtype=torch.float64, device="cuda")
        out = np.zeros((N_MOVES, wl.n_bins))
        for i in range(N_MOVES):
            bps.bps_hmc_step(s.ctx, False)
            bps.bps_get_spectrum(s.ctx, spec)
            bps.bps_bin_power_noalloc(N, wl.box, wl.n_bins, spec, sig)
            out[i] = sig.cpu().numpy()
    finally:
        s.close()
    x = np.log(out)
    ess = np.array([diagnostics.ess_geyer(x[:, m]) for m in range(x.shape[1])])
    return x.mean(0), x.std(0), ess


def test_network_predicts_held_out_multipliers(trained):
    pc, F, T = trained
    err = np.sqrt(np.mean((pc.predict_log(F) - T) ** 2))
    plain = np.sqrt(np.mean(T ** 2))
    assert err < 0.6 * plain, (err, plain)


def test_network_mass_raises_the_effective_sample_size(trained):
    pc, _, _ = trained
    m0, s0, e0 = chain_stats(None, 0.15, 5)
    m1, s1, e1 = chain_stats(pc, 0.15, 5)
    print("ESS plain", np.round(e0).tolist(), "network", np.round(e1).tolist())
    assert e1.min() > 2.0 * e0.min(), (e0, e1)
    assert np.all(e1[:2] > 3.0 * e0[:2]), (e0, e1)
    se = np.sqrt(s0 ** 2 / e0 + s1 ** 2 / e1)
    assert np.all(np.abs(m1 - m0) < 5.0 * se), (m0, m1, se)
