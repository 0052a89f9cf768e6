"""The preconditioner's inputs and its effect on the HMC move, against the FP64
oracle: the window power feature, the mode statistics the targets are built
from, and HMC moves under a scaled diagonal mass (mass_mode 1).

Tolerances: window power relative 1e-5 per bin (FP32 transform of a, FP64 bin
sums); mode statistics relative 1e-3 per bin (differences of FP64 sums of FP32
states that agree to 2e-4 in relative L2); scaled-mass HMC as in the
unscaled parity test."""
import math

import numpy as np
import pytest

from oracle import grid, hmc, model
from tests.helpers import Problem, gpu_spectrum, rel_l2

pytestmark = pytest.mark.gpu


def sampler(pb, seed, mass_mode):
    import torch

    from paper_1306_1821_gb300 import bps
    kw = pb.config_kwargs(seed)
    s = bps.Sampler(pb.N, pb.wl.box, pb.wl.n_sub, pb.wl.n_bins, mass_mode=mass_mode, **kw)
    bps.bps_set_data(s.ctx, torch.from_numpy(pb.counts).cuda(), torch.from_numpy(pb.R).cuda())
    bps.bps_set_state(s.ctx, None, pb.P, pb.b, pb.nbar, 0)
    bps.bps_set_spectrum(s.ctx, torch.from_numpy(pb.dh32).cuda())
    return s


@pytest.mark.parametrize("N,n_sub", [(16, 1), (32, 3)])
def test_window_power_matches_oracle(N, n_sub):
    from oracle import gibbs
    from paper_1306_1821_gb300 import bps
    pb = Problem(N, n_sub=n_sub, n_bins=6)
    s = sampler(pb, 5, 0)
    try:
        got = bps.bps_window_power(s.ctx, pb.wl.n_bins)[0]
    finally:
        s.close()
    a, _ = model.local_fields(pb.counts, pb.R, pb.b, pb.nbar)
    ref = gibbs.bin_power(pb.geom, grid.forward(a / a.mean()))
    assert np.max(np.abs(got / ref - 1)) < 1e-5


def test_mode_statistics_match_oracle_chain():
    from paper_1306_1821_gb300 import bps
    pb = Problem(16, n_sub=2, n_bins=4, n_leapfrog=6, eps_max=0.1)
    n_mass, S = 3, 5
    s = sampler(pb, 31, 0)
    try:
        V, Mb = bps.bps_mass_stats(s.ctx, S, n_mass)
        _, _, _, it = bps.bps_get_state(s.ctx, None, pb.wl.n_bins, pb.wl.n_sub)
    finally:
        s.close()
    assert it == S
    ch = pb.oracle_chain(seed=31)
    states, n_acc = [], 0
    for _ in range(S):
        info = ch.hmc_step()
        ch.iteration += 1
        if abs(info["dH"] + math.log(info["u_acc"])) < 1e-3:
            pytest.skip("decision within the tolerance band; states may legitimately differ")
        states.append(ch.delta_hat.copy())
        n_acc += info["accepted"]
    assert n_acc >= 3          # the states differ, so the variances are not rounding noise
    X = np.stack(states)
    var_k = np.mean(np.abs(X) ** 2, 0) - np.abs(X.mean(0)) ** 2        # per-mode sample variance
    gm = grid.Geometry(16, pb.wl.box, n_mass)
    M, _ = model.mass_diag(pb.geom, pb.P, ch.abar)
    for j in range(n_mass):
        sel = gm.bin == j
        w = pb.geom.w[sel]
        v_ref = np.sum(w * var_k[sel]) / np.sum(w) / pb.geom.Nv
        m_ref = np.sum(w * M[sel]) / np.sum(w)
        assert V[0, j] == pytest.approx(v_ref, rel=1e-3)
        assert Mb[0, j] == pytest.approx(m_ref, rel=1e-6)     # abar from the FP32 field a


@pytest.mark.parametrize("N,n_sub", [(16, 1), (32, 2)])
def test_scaled_mass_hmc_matches_oracle(N, n_sub):
    from paper_1306_1821_gb300 import bps
    pb = Problem(N, n_sub=n_sub, n_bins=4, n_leapfrog=6, eps_max=0.4)
    scales = np.array([0.45, 1.7, 0.9, 2.5, 0.6])
    s = sampler(pb, 23, 1)
    try:
        bps.bps_set_mass_scale(s.ctx, scales)
        ch = pb.oracle_chain(seed=23)
        gm = grid.Geometry(N, pb.wl.box, scales.size)
        per_mode = gm.per_mode(scales, dc=1.0)
        for it in range(3):
            acc, dH, eps = bps.bps_hmc_step(s.ctx)
            d1, info = hmc.hmc_move(pb.geom, ch.delta_hat, ch.P, ch.a, ch.c, ch.abar, ch.n_leapfrog, ch.eps_max,
                                    ch.seed, ch.iteration, mass_scale=per_mode)
            ch.delta_hat = d1
            ch.iteration += 1
            assert eps == pytest.approx(info["eps"], rel=1e-15)
            assert abs(dH - info["dH"]) < 1e-3, (dH, info["dH"])
            if abs(info["dH"] + math.log(info["u_acc"])) < 1e-3:
                pytest.skip("decision within the tolerance band; states may legitimately differ")
            assert bool(acc) == info["accepted"]
            assert rel_l2(gpu_spectrum(s), ch.delta_hat) < 2e-4
    finally:
        s.close()


def test_unit_scales_equal_the_plain_mass():
    from paper_1306_1821_gb300 import bps
    pb = Problem(16, n_sub=1, n_bins=4, n_leapfrog=6, eps_max=0.4)
    a = sampler(pb, 9, 0)
    b = sampler(pb, 9, 1)
    try:
        bps.bps_set_mass_scale(b.ctx, np.ones(7))
        for _ in range(2):
            ra = bps.bps_hmc_step(a.ctx)
            rb = bps.bps_hmc_step(b.ctx)
            assert ra == rb
        assert np.array_equal(gpu_spectrum(a), gpu_spectrum(b))
    finally:
        a.close()
        b.close()


def oracle_net_scales(params, P, W, mu, sd, clamp):
    """exp(clamp(net(z))) of the oracle network with BF16-rounded operands."""
    from oracle import mlp
    f = np.concatenate([np.log(P), np.log(W)]).astype(np.float32).astype(np.float64)
    z = np.clip(((f - mu) / sd).astype(np.float32), -4, 4).astype(np.float64)
    y, _ = mlp.forward(params, z[None, :], mlp.round_bf16)
    return np.exp(np.clip(y[0], -clamp, clamp))


def random_net(n_in, n_out, seed):
    from oracle import mlp
    from paper_1306_1821_gb300 import bps
    rng = np.random.default_rng(seed)
    sizes = [n_in, 32, 32, n_out]
    params = mlp.init_params(sizes, seed)
    for i in range(1, len(params), 2):
        params[i] = rng.standard_normal(params[i].shape) * 0.1
    params[-2] *= 0.3
    net = bps.MLP(sizes)
    net.set_params(bps.flatten_params(params))
    p32 = bps.unflatten_params(net.get_params(), sizes)
    mu = rng.standard_normal(n_in).astype(np.float32)
    sd = rng.uniform(0.5, 2.0, n_in).astype(np.float32)
    return net, p32, mu.astype(np.float64), sd.astype(np.float64)


def test_network_mass_is_evaluated_on_the_device_from_the_current_state():
    from oracle import gibbs
    from paper_1306_1821_gb300 import bps
    pb = Problem(16, n_sub=2, n_bins=4, n_leapfrog=6, eps_max=0.1)
    n_mass, clamp = 5, np.log(16.0)
    net, p32, mu, sd = random_net(8, n_mass, 3)
    s = sampler(pb, 41, 0)
    try:
        bps.bps_set_mass_net(s.ctx, net, mu, sd, clamp)
        net.close()                       # the context holds its own copy
        a, _ = model.local_fields(pb.counts, pb.R, pb.b, pb.nbar)
        W = gibbs.bin_power(pb.geom, grid.forward(a / a.mean()))
        for _ in range(2):
            bps.bps_gibbs_iterate(s.ctx, 1)
            P, _, _, _ = bps.bps_get_state(s.ctx, None, pb.wl.n_bins, pb.wl.n_sub)
            bps.bps_hmc_step(s.ctx)           # scales from the P after the iteration
            got = bps.bps_get_mass_scale(s.ctx)
            assert got.size == n_mass
            ref = oracle_net_scales(p32, P[:4], W, mu, sd, clamp)
            assert np.max(np.abs(np.log(got / ref))) < 5e-3, (got, ref)
        bps.bps_set_mass_net(s.ctx, None)
    finally:
        s.close()


def test_gibbs_with_network_mass_matches_oracle_chain():
    from oracle import gibbs
    from paper_1306_1821_gb300 import bps
    pb = Problem(16, n_sub=2, n_bins=4, n_leapfrog=6, eps_max=0.3)
    n_mass, clamp = 6, np.log(16.0)
    net, p32, mu, sd = random_net(8, n_mass, 8)
    s = sampler(pb, 43, 0)
    try:
        bps.bps_set_mass_net(s.ctx, net, mu, sd, clamp)
        ch = pb.oracle_chain(seed=43)
        a, _ = model.local_fields(pb.counts, pb.R, pb.b, pb.nbar)
        W = gibbs.bin_power(pb.geom, grid.forward(a / a.mean()))
        gm = grid.Geometry(16, pb.wl.box, n_mass)
        ch.mass_fn = lambda c: gm.per_mode(oracle_net_scales(p32, c.P, W, mu, sd, clamp), dc=1.0)
        rec = bps.bps_gibbs_iterate(s.ctx, 3, rec_len=4 + 2 * 2 + 2)
        for i in range(3):
            r = ch.iterate()
            if abs(r["hmc"]["dH"] + math.log(r["hmc"]["u_acc"])) < 1e-3:
                pytest.skip("decision within the tolerance band; states may legitimately differ")
            assert abs(rec[i, -2] - r["hmc"]["dH"]) < 1e-3
            assert bool(rec[i, -1]) == r["hmc"]["accepted"]
            assert np.max(np.abs(rec[i, :4] / r["P"] - 1)) < 1e-4
        assert rel_l2(gpu_spectrum(s), ch.delta_hat) < 2e-4
    finally:
        net.close()
        s.close()


def test_invalid_preconditioner_arguments_are_rejected():
    from paper_1306_1821_gb300 import bps
    pb = Problem(16, n_sub=1, n_bins=4)
    s = sampler(pb, 3, 0)
    try:
        with pytest.raises(bps.BpsError):
            bps.bps_mass_stats(s.ctx, 2, 60)                 # a mass bin with no mode at 16^3
        with pytest.raises(bps.BpsError):
            bps.bps_set_mass_scale(s.ctx, np.array([1.0, -2.0]))
        net = bps.MLP([7, 8, 5])                              # input width must be 2 n_bins = 8
        try:
            with pytest.raises(bps.BpsError):
                bps.bps_set_mass_net(s.ctx, net, np.zeros(7), np.ones(7), 2.0)
        finally:
            net.close()
        net = bps.MLP([8, 8, 5])
        try:
            with pytest.raises(bps.BpsError):
                bps.bps_set_mass_net(s.ctx, net, np.zeros(8), np.zeros(8), 2.0)   # zero feature scale
            bps.bps_set_mass_net(s.ctx, net, np.zeros(8), np.ones(8), 2.0)
            with pytest.raises(bps.BpsError):
                bps.bps_mass_stats(s.ctx, 2, 3)                  # must equal the network's 5 outputs
        finally:
            net.close()
    finally:
        s.close()
    with pytest.raises(bps.BpsError):
        bps.MLP([8, 0, 5])
    with pytest.raises(bps.BpsError):
        bps.MLP([8, 8, 8, 8, 8, 8])                            # more than four layers


def test_saved_preconditioner_installs_identically(tmp_path):
    from paper_1306_1821_gb300 import bps, precond
    pb = Problem(16, n_sub=1, n_bins=4, n_leapfrog=6, eps_max=0.2)
    net, p32, mu, sd = random_net(8, 5, 17)
    a = sampler(pb, 7, 0)
    b = sampler(pb, 7, 0)
    try:
        bps.bps_set_mass_net(a.ctx, net, mu, sd, np.log(16.0))
        blob = bps.bps_mlp_export(net, mu, sd, np.log(16.0))
        path = tmp_path / "mass.bpsm"
        path.write_bytes(blob)
        precond.install_saved(b.ctx, str(path))
        for _ in range(2):
            assert bps.bps_hmc_step(a.ctx) == bps.bps_hmc_step(b.ctx)
        assert np.array_equal(bps.bps_get_mass_scale(a.ctx), bps.bps_get_mass_scale(b.ctx))
        with pytest.raises(bps.BpsError):
            bps.bps_set_preconditioner(b.ctx, blob[:-4])
        with pytest.raises(bps.BpsError):
            bps.bps_set_preconditioner(b.ctx, b"XXXX" + blob[4:])
    finally:
        net.close()
        a.close()
        b.close()
