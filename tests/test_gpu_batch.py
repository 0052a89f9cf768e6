"""Batches of independent chains on uneven grids: every chain of a batch must
follow its own FP64 oracle chain (through the C ABI), and equal a single-chain
context run with the same key."""
import numpy as np
import pytest

from oracle import gibbs, grid
from paper_1306_1821_gb300 import inputs
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu

SIZES = [16, 32, 16, 32]
NSUB = [1, 2, 2, 1]


def problems():
    out = []
    for j, (N, ns) in enumerate(zip(SIZES, NSUB)):
        wl = inputs.small_workload(N, n_bins=3, n_sub=ns, f_sky=0.6, seed=40 + j)
        delta, counts, R = inputs.make_survey(wl)
        d32 = (0.8 * delta).astype(np.float32)
        out.append((wl, counts, R, d32))
    return out


def config(bps, seed):
    return bps.make_config(3, n_leapfrog=5, eps_max=0.25, jump=1, jump_leapfrog=3, jump_eps_max=0.2,
                           fixed_bias_index=0, seed=seed)


def test_batch_chains_match_their_oracles():
    import torch

    from paper_1306_1821_gb300 import bps
    ps = problems()
    cfg = config(bps, 100)
    batch = bps.bps_create_batch(SIZES, [p[0].box for p in ps], NSUB, cfg)
    try:
        for j, (wl, counts, R, d32) in enumerate(ps):
            P, b, nbar = inputs.initial_state(wl)
            bps.bps_batch_set_chain(batch, j, torch.from_numpy(counts).cuda(), torch.from_numpy(R).cuda(),
                                    torch.from_numpy(d32).cuda(), P, b, nbar, 0)
        n_iter = 2
        rec = bps.bps_batch_gibbs_iterate(batch, n_iter, len(ps))
        for j, (wl, counts, R, d32) in enumerate(ps):
            P, b, nbar = inputs.initial_state(wl)
            g = grid.Geometry(wl.N, wl.box, 3)
            dh = grid.forward(d32.astype(np.float64))
            dh[0, 0, 0] = 0
            ch = gibbs.Chain(g, counts, R, P, b, nbar, delta_hat=dh, n_leapfrog=5, eps_max=0.25, jump=True,
                             jump_leapfrog=3, jump_eps_max=0.2, fixed_bias=0, seed=100 + j)
            slot = bps.bps_batch_record_slot(batch, j)
            ns = wl.n_sub
            for i in range(n_iter):
                r = ch.iterate()
                got = rec[i, slot]
                assert np.max(np.abs(got[:3] / r["P"] - 1)) < 1e-4, (j, i)
                assert np.max(np.abs(got[3:3 + ns] - r["b"])) < 1e-3
                assert np.max(np.abs(got[3 + ns:3 + 2 * ns] / r["nbar"] - 1)) < 1e-4
                assert abs(got[3 + 2 * ns] - r["hmc"]["dH"]) < 1e-3
            Pg, bg, ng, it = bps.bps_batch_get_chain(batch, j, None, 3, ns)
            assert it == n_iter
            assert np.allclose(Pg[:3], ch.P, rtol=1e-4)
            # the chain's field after the iterations
            out = torch.zeros((wl.N,) * 3, dtype=torch.float32, device="cuda")
            bps.bps_batch_get_chain(batch, j, out, 3, ns)
            assert rel_l2(out.cpu().numpy(), grid.inverse(ch.delta_hat, wl.N)) < 2e-4
    finally:
        bps.bps_destroy(batch)


def test_batch_chain_equals_single_context():
    import torch

    from paper_1306_1821_gb300 import bps
    ps = problems()
    cfg = config(bps, 7)
    batch = bps.bps_create_batch(SIZES, [p[0].box for p in ps], NSUB, cfg)
    try:
        for j, (wl, counts, R, d32) in enumerate(ps):
            P, b, nbar = inputs.initial_state(wl)
            bps.bps_batch_set_chain(batch, j, torch.from_numpy(counts).cuda(), torch.from_numpy(R).cuda(),
                                    torch.from_numpy(d32).cuda(), P, b, nbar, 0)
        rec = bps.bps_batch_gibbs_iterate(batch, 3, len(ps))
        for j in (1, 2):
            wl, counts, R, d32 = ps[j]
            P, b, nbar = inputs.initial_state(wl)
            s = bps.Sampler(wl.N, wl.box, wl.n_sub, 3, n_leapfrog=5, eps_max=0.25, jump=1, jump_leapfrog=3,
                            jump_eps_max=0.2, fixed_bias_index=0, seed=7 + j)
            bps.bps_set_data(s.ctx, torch.from_numpy(counts).cuda(), torch.from_numpy(R).cuda())
            bps.bps_set_state(s.ctx, torch.from_numpy(d32).cuda(), P, b, nbar, 0)
            single = bps.bps_gibbs_iterate(s.ctx, 3, s.rec_len)
            slot = bps.bps_batch_record_slot(batch, j)
            L = s.rec_len
            assert np.allclose(rec[:, slot, :L], single, rtol=1e-5, atol=1e-6)
            s.close()
    finally:
        bps.bps_destroy(batch)


def test_batch_with_network_mass_equals_single_contexts():
    import torch

    from oracle import mlp
    from paper_1306_1821_gb300 import bps
    ps = problems()
    sizes = [6, 16, 16, 4]                       # 2 n_bins inputs (3 bins), 4 mass bins
    net = bps.MLP(sizes)
    rng = np.random.default_rng(3)
    params = mlp.init_params(sizes, 4)
    for i in range(1, len(params), 2):
        params[i] = rng.standard_normal(params[i].shape) * 0.1
    net.set_params(bps.flatten_params(params))
    mu, sd = rng.standard_normal(6), rng.uniform(0.5, 2.0, 6)
    cfg = config(bps, 70)
    batch = bps.bps_create_batch(SIZES, [p[0].box for p in ps], NSUB, cfg)
    try:
        for j, (wl, counts, R, d32) in enumerate(ps):
            P, b, nbar = inputs.initial_state(wl)
            bps.bps_batch_set_chain(batch, j, torch.from_numpy(counts).cuda(), torch.from_numpy(R).cuda(),
                                    torch.from_numpy(d32).cuda(), P, b, nbar, 0)
        bps.bps_set_mass_net(batch, net, mu, sd, np.log(16.0))
        rec = bps.bps_batch_gibbs_iterate(batch, 2, len(ps))
        for j in (0, 3):
            wl, counts, R, d32 = ps[j]
            P, b, nbar = inputs.initial_state(wl)
            s = bps.Sampler(wl.N, wl.box, wl.n_sub, 3, n_leapfrog=5, eps_max=0.25, jump=1, jump_leapfrog=3,
                            jump_eps_max=0.2, fixed_bias_index=0, seed=70 + j)
            bps.bps_set_data(s.ctx, torch.from_numpy(counts).cuda(), torch.from_numpy(R).cuda())
            bps.bps_set_state(s.ctx, torch.from_numpy(d32).cuda(), P, b, nbar, 0)
            bps.bps_set_mass_net(s.ctx, net, mu, sd, np.log(16.0))
            single = bps.bps_gibbs_iterate(s.ctx, 2, s.rec_len)
            slot = bps.bps_batch_record_slot(batch, j)
            assert np.allclose(rec[:, slot, :s.rec_len], single, rtol=1e-5, atol=1e-6)
            assert np.allclose(bps.bps_get_mass_scale(batch, j), bps.bps_get_mass_scale(s.ctx), rtol=1e-6)
            s.close()
    finally:
        bps.bps_destroy(batch)
        net.close()


def test_batch_of_the_96_chain_workload_sizes_matches_oracles():
    """Chains drawn from the 96-chain batch workload (32^3, 64^3 and 96^3 grids,
    caps of 20-60% of the sky with linear fall-off, 3-4 subsamples, 16 bins,
    jump on): two Gibbs iterations of each against its own oracle chain, the
    96^3 chains taking the radix-3 transform path inside the batch."""
    import torch

    from paper_1306_1821_gb300 import bps
    from tests.helpers import compare_chain
    wls = inputs.batch_workloads()
    pick = [wls[j] for j in (3, 32, 34, 66, 67)]
    cfg = bps.make_config(16, n_leapfrog=10, eps_max=0.1, jump=1, jump_leapfrog=4, jump_eps_max=0.2,
                          fixed_bias_index=0, seed=500)
    batch = bps.bps_create_batch([w.N for w in pick], [w.box for w in pick], [w.n_sub for w in pick], cfg)
    try:
        starts = []
        for j, wl in enumerate(pick):
            delta, counts, R = inputs.make_survey(wl)
            d32 = (0.8 * delta).astype(np.float32)
            P, b, nbar = inputs.initial_state(wl)
            bps.bps_batch_set_chain(batch, j, torch.from_numpy(counts).cuda(), torch.from_numpy(R).cuda(),
                                    torch.from_numpy(d32).cuda(), P, b, nbar, 0)
            starts.append((counts, R, d32, P, b, nbar))
        n_iter = 2
        rec = bps.bps_batch_gibbs_iterate(batch, n_iter, len(pick))
        for j, wl in enumerate(pick):
            counts, R, d32, P, b, nbar = starts[j]
            g = grid.Geometry(wl.N, wl.box, 16)
            dh = grid.forward(d32.astype(np.float64))
            dh[0, 0, 0] = 0
            ch = gibbs.Chain(g, counts, R, P, b, nbar, delta_hat=dh, n_leapfrog=10, eps_max=0.1, jump=True,
                             jump_leapfrog=4, jump_eps_max=0.2, fixed_bias=0, seed=500 + j)
            slot = bps.bps_batch_record_slot(batch, j)
            L = 16 + 2 * wl.n_sub + 2
            done, worst = compare_chain(rec[:, slot, :L], ch, n_iter)
            assert done >= 1, (j, wl.N)
    finally:
        bps.bps_destroy(batch)
