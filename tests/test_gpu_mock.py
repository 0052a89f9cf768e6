"""Artificial surveys generated on the device (Sec. 5; App. D; Eq. rel_bias),
through the C ABI, against the FP64 oracle (oracle/mock.py).

  * Field: relative L2 <= 1e-5 against the FP64 field from the same Philox
    normals (FP32 normals and transforms against FP64), 32^3 to 256^3.
  * Counts: bit-exact.  Both sides take every decision in FP64 from the same
    inputs (the device's FP32 field and response) with IEEE-exact operations;
    the Gaussian form uses log and cos, so a count may differ only where
    x = mean + sd z lies within 1e-9 of a half-integer (none is expected).
  * Response: bit-exact (the same FP64 geometry and interpolation).
  * The paper's fifteen luminosity subsamples (Sec. 5): Schechter selection and
    mean numbers per magnitude bin, bias law, a 128^3 survey made on the
    device, and Gibbs iterations of the sampler on it against the oracle chain.
"""
import numpy as np
import pytest

from oracle import mock
from paper_1306_1821_gb300 import inputs
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


def spectrum_table(N, box):
    n2 = np.arange(3 * (N // 2) ** 2 + 1, dtype=np.float64)
    k = 2.0 * np.pi * np.sqrt(n2) / box
    P = inputs.true_spectrum(k, N, box)
    P[0] = 0.0
    return P


def sampler(N, box, n_sub, n_bins=8):
    from paper_1306_1821_gb300 import bps
    return bps.Sampler(N, box, n_sub, n_bins, n_leapfrog=5, eps_max=0.1, seed=1)


@pytest.mark.parametrize("N", [32, 96, 128, 256])
def test_mock_field_matches_oracle(N):
    import torch

    from paper_1306_1821_gb300 import bps
    box = 500.0 * N / 32
    s = sampler(N, box, 1)
    try:
        P = spectrum_table(N, box)
        d = torch.zeros((N, N, N), dtype=torch.float32, device="cuda")
        bps.bps_mock_field(s.ctx, 77, P, d)
        torch.cuda.synchronize()
        amp = np.sqrt(P / (box / N) ** 3)
        ref = mock.field(N, amp, 77)
        assert rel_l2(d.cpu().numpy(), ref) < 1e-5
    finally:
        s.close()


def survey_on_device(s, N, box, seed, table, f_sky, axis, b, nbar, noise):
    import torch

    from paper_1306_1821_gb300 import bps
    n_sub = len(b)
    d = torch.zeros((N, N, N), dtype=torch.float32, device="cuda")
    bps.bps_mock_field(s.ctx, seed, spectrum_table(N, box), d)
    R = torch.zeros((n_sub, N, N, N), dtype=torch.float32, device="cuda")
    bps.bps_mock_response(s.ctx, f_sky, axis, table, R)
    c = torch.zeros((n_sub, N, N, N), dtype=torch.int32, device="cuda")
    bps.bps_mock_counts(s.ctx, seed, d, R, b, nbar, noise, c)
    torch.cuda.synchronize()
    return d, R, c


@pytest.mark.parametrize("noise", [0, 1])
def test_mock_counts_and_response_bit_exact(noise):
    from paper_1306_1821_gb300 import bps
    N, box, n_sub = 64, 750.0, 3
    edges = np.array([-22.0, -21.0, -20.0, -19.0])
    table, nb_rel = bps.bps_schechter_tables(edges, box / 2, 257)
    b = bps.bps_bias_law(0.5 * (edges[:-1] + edges[1:]))
    nbar = 6.0 * nb_rel / nb_rel.max()
    axis = (0.3, -0.4, 0.87)
    s = sampler(N, box, n_sub)
    try:
        d, R, c = survey_on_device(s, N, box, 123, table, 0.35, axis, b, nbar, noise)
        Rg = R.cpu().numpy()
        Rref = mock.response(N, box, 0.35, axis, table, box / 2)
        assert np.array_equal(Rg.view(np.uint32), Rref.view(np.uint32))
        dg = d.cpu().numpy()
        cg = c.cpu().numpy()
        if noise == 0:
            ref = mock.counts(dg, Rg, b, nbar, 123, "poisson")
            assert np.array_equal(cg, ref)
        else:
            ref = mock.counts(dg, Rg, b, nbar, 123, "gauss")
            for l in range(n_sub):
                # a count may differ only where mean + sd z lies at a rounding tie
                # (log and cos are not correctly rounded on either side)
                diff = cg[l] != ref[l]
                assert diff.sum() <= 2, diff.sum()
                if diff.any():
                    assert np.all(np.abs(np.abs(cg[l][diff] - ref[l][diff])) == 1)
        assert cg.sum() > 0
    finally:
        s.close()


def test_mock_survey_at_full_size_sampled():
    """256^3, six subsamples of the benchmark survey: field within 1e-5, counts
    bit-exact on 40000 sampled voxels per subsample (oracle from the device's
    own FP32 field and response)."""
    import torch

    from paper_1306_1821_gb300 import bps
    wl = inputs.WORKLOADS["survey256"]
    N, box = wl.N, wl.box
    Rh = inputs.response(N, box, wl.f_sky, wl.radial, wl.r0)
    s = sampler(N, box, wl.n_sub, 32)
    try:
        d = torch.zeros((N, N, N), dtype=torch.float32, device="cuda")
        bps.bps_mock_field(s.ctx, 5, spectrum_table(N, box), d)
        R = torch.from_numpy(np.broadcast_to(Rh, (wl.n_sub, N, N, N)).copy()).cuda()
        c = torch.zeros((wl.n_sub, N, N, N), dtype=torch.int32, device="cuda")
        bps.bps_mock_counts(s.ctx, 5, d, R, wl.b, wl.nbar, 0, c)
        torch.cuda.synchronize()
        dg = d.cpu().numpy().ravel()
        rng = np.random.default_rng(0)
        obs = np.nonzero(Rh.ravel() > 0)[0]
        idx = np.sort(rng.choice(obs, 40000, replace=False))
        cg = c.cpu().numpy().reshape(wl.n_sub, -1)
        for l in range(wl.n_sub):
            lam = mock.mean_counts(dg[idx], Rh.ravel()[idx], wl.b[l], wl.nbar[l])
            ref = mock.poisson_counts(lam, 5, l, index=idx)
            assert np.array_equal(cg[l, idx], ref)
        assert np.all(cg[:, Rh.ravel() == 0] == 0)
    finally:
        s.close()


def test_fifteen_subsample_schechter_survey_and_chain():
    """The paper's setup (Sec. 5): fifteen absolute-magnitude bins from -23 to
    -17, the Schechter selection and mean numbers per bin, the bias law, a 25%
    cap; survey made on the device, then three Gibbs iterations (jump on) of
    the sampler against the oracle chain on the same data."""
    import torch

    from paper_1306_1821_gb300 import bps
    from tests.helpers import Problem, compare_chain
    wl = inputs.WORKLOADS["schechter128"]
    N, box = wl.N, wl.box
    edges = np.asarray(wl.extra["M_edges"])
    table, nb_rel = bps.bps_schechter_tables(edges, box / 2, 1025)
    assert np.allclose(nb_rel * wl.extra["phi_star"], wl.nbar, rtol=1e-11)
    assert np.allclose(bps.bps_bias_law(0.5 * (edges[:-1] + edges[1:])), wl.b, rtol=1e-14)
    s = sampler(N, box, wl.n_sub, wl.n_bins)
    try:
        d, R, c = survey_on_device(s, N, box, 9, table, wl.f_sky, (0, 0, 1), wl.b, wl.nbar, 0)
        counts, Rg = c.cpu().numpy(), R.cpu().numpy()
    finally:
        s.close()
    assert counts.max() <= 65535 and counts.sum() > 0
    assert np.all((Rg > 0).reshape(wl.n_sub, -1).any(1))      # every subsample observes some voxels
    pb = Problem(N, wl=wl, survey=(d.cpu().numpy().astype(np.float64), counts.astype(np.int32), Rg))
    g = pb.gpu(seed=41, jump=1)
    try:
        rec = bps.bps_gibbs_iterate(g.ctx, 3, g.rec_len)
        done, worst = compare_chain(rec, pb.oracle_chain(seed=41, jump=True), 3)
        print(f"15 subsamples: {done} iterations compared, max |dH - dH_oracle| = {worst:.2e}")
        assert done >= 2
    finally:
        g.close()
