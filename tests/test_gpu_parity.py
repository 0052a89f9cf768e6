"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP32 fields against FP64, from the FP32 rounding of each step):
  * 3D transforms: relative L2 <= 2e-6 (FP32 rounding of log2(N^3) butterfly stages);
  * force (Eq. Wiener_Posterior_force): relative L2 <= 1e-5;
  * HMC move: |dH_gpu - dH_oracle| <= 1e-3 and the same Metropolis decision unless
    |dH + ln u| < 1e-3; end state relative L2 <= 2e-4;
  * k-bin power sigma_m: relative <= 2e-6 per bin;
  * Philox words: bit-exact; momentum normals: |diff| <= 2e-6 (FP32 transform).
"""
import math

import numpy as np
import pytest

from oracle import gibbs, grid, hmc, model, philox
from tests.helpers import Problem, gpu_spectrum, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    from paper_1306_1821_gb300 import bps
    bps.load()
    return torch


def test_library_loads(torch_cuda):
    from paper_1306_1821_gb300 import bps
    assert "sm_103a" in bps.bps_version()


def test_philox_words_bit_exact(torch_cuda):
    from paper_1306_1821_gb300 import bps
    torch = torch_cuda
    for (seed, it, stage, sub, blk0, n) in [(0, 0, 1, 0, 0, 64), (2**63 + 11, 7, 3, 5, 1000, 37), (5, 2**40, 6, 1, 2**50, 9)]:
        out = torch.zeros(n, dtype=torch.int64, device="cuda")
        bps.bps_philox_words(seed, it, stage, sub, blk0, out)
        got = out.cpu().numpy().view(np.uint64)
        blocks = blk0 + np.arange((n + 3) // 4, dtype=np.uint64)
        w = philox.words(seed, it, stage, sub, blocks)
        ref = np.stack(w, 1).ravel()[:n]
        assert np.array_equal(got, ref)


def test_voxel_normals_match_oracle(torch_cuda):
    from paper_1306_1821_gb300 import bps
    torch = torch_cuda
    n = (1 << 20) + 5
    out = torch.zeros(n, dtype=torch.float32, device="cuda")
    bps.bps_voxel_normals(77, 3, out)
    got = out.cpu().numpy().astype(np.float64)
    ref = philox.voxel_normals(77, 3, philox.STAGE_MOMENTUM, 0, n)
    assert np.max(np.abs(got - ref)) < 2e-6


@pytest.mark.parametrize("N", [8, 16, 32, 64, 96, 128])
def test_fft_roundtrip_against_numpy(torch_cuda, N):
    from paper_1306_1821_gb300 import bps
    torch = torch_cuda
    cfg = bps.make_config(2 if N >= 8 else 1)
    ctx = bps.bps_create(N, 100.0, 1, cfg)
    try:
        rng = np.random.default_rng(N)
        x = rng.standard_normal((N, N, N)).astype(np.float32)
        xs = torch.from_numpy(x).cuda()
        spec = torch.zeros((N, N, N // 2 + 1), dtype=torch.complex64, device="cuda")
        bps.bps_fft_r2c(ctx, xs, spec)
        ref = np.fft.rfftn(x.astype(np.float64))
        assert rel_l2(spec.cpu().numpy(), ref) < 2e-6
        back = torch.zeros_like(xs)
        # inverse of an exact (FP64-rounded) spectrum
        bps.bps_fft_c2r(ctx, torch.from_numpy(ref.astype(np.complex64)).cuda(), back)
        assert rel_l2(back.cpu().numpy(), x.astype(np.float64)) < 2e-6
    finally:
        bps.bps_destroy(ctx)


@pytest.mark.parametrize("N,n_sub", [(16, 1), (32, 2), (64, 3), (96, 2), (128, 2), (256, 1)])
def test_gradient_and_energies(torch_cuda, N, n_sub):
    from paper_1306_1821_gb300 import bps
    torch = torch_cuda
    pb = Problem(N, n_sub=n_sub, n_bins=4)
    s = pb.gpu()
    try:
        g = torch.zeros((N, N, N // 2 + 1), dtype=torch.complex64, device="cuda")
        e = bps.bps_gradient(s.ctx, g)
        a, c = model.local_fields(pb.counts, pb.R, pb.b, pb.nbar)
        gh, lik = model.gradient_hat(pb.geom, pb.dh, pb.P, a, c)
        assert rel_l2(g.cpu().numpy(), gh) < 1e-5
        prior = model.prior_energy(pb.geom, pb.dh, pb.P)
        assert e[0] == pytest.approx(prior, rel=1e-5)
        assert abs(e[1] - lik) < 1e-5 * (abs(lik) + np.sum(np.abs(a * grid.inverse(pb.dh, N) ** 2)))
    finally:
        s.close()


@pytest.mark.parametrize("N,n_sub,f_sky", [(32, 2, 0.6), (64, 3, 0.25), (128, 2, 0.4)])
def test_gradient_three_passes_with_line_supports(torch_cuda, monkeypatch, N, n_sub, f_sky):
    """The force z pass stages a and c only on each z line's support (R > 0 in some
    subsample) and writes a zero force on tiles without support; grids up to 128^3
    normally take the fused plane kernel, so the three passes are forced here.  A
    support that missed an observed voxel would drop its a and c from the force."""
    from paper_1306_1821_gb300 import bps
    monkeypatch.setenv("BPS_FUSED_YZ", "0")
    torch = torch_cuda
    pb = Problem(N, n_sub=n_sub, n_bins=4, f_sky=f_sky)
    assert (pb.R.reshape(n_sub, -1).max(0) == 0).mean() > 0.3   # a survey with unobserved lines
    s = pb.gpu()
    try:
        g = torch.zeros((N, N, N // 2 + 1), dtype=torch.complex64, device="cuda")
        e = bps.bps_gradient(s.ctx, g)
        a, c = model.local_fields(pb.counts, pb.R, pb.b, pb.nbar)
        gh, lik = model.gradient_hat(pb.geom, pb.dh, pb.P, a, c)
        assert rel_l2(g.cpu().numpy(), gh) < 1e-5
        assert abs(e[1] - lik) < 1e-5 * (abs(lik) + np.sum(np.abs(a * grid.inverse(pb.dh, N) ** 2)))
    finally:
        s.close()


def test_line_supports_follow_new_data(torch_cuda, monkeypatch):
    """Uploading a second survey with a wider mask into the same context resets the
    per-line supports: the force then matches the oracle on the new survey."""
    from paper_1306_1821_gb300 import bps
    monkeypatch.setenv("BPS_FUSED_YZ", "0")
    torch = torch_cuda
    N = 64
    narrow = Problem(N, n_sub=2, n_bins=4, f_sky=0.15, seed=5)
    wide = Problem(N, n_sub=2, n_bins=4, f_sky=0.9, seed=6)
    s = narrow.gpu()
    try:
        bps.bps_set_data(s.ctx, torch.from_numpy(wide.counts).cuda(), torch.from_numpy(wide.R).cuda())
        bps.bps_set_state(s.ctx, None, wide.P, wide.b, wide.nbar, 0)
        bps.bps_set_spectrum(s.ctx, torch.from_numpy(wide.dh32).cuda())
        g = torch.zeros((N, N, N // 2 + 1), dtype=torch.complex64, device="cuda")
        bps.bps_gradient(s.ctx, g)
        a, c = model.local_fields(wide.counts, wide.R, wide.b, wide.nbar)
        gh, _ = model.gradient_hat(wide.geom, wide.dh, wide.P, a, c)
        assert rel_l2(g.cpu().numpy(), gh) < 1e-5
    finally:
        s.close()


@pytest.mark.parametrize("N,n_sub,moves", [(16, 1, 4), (32, 2, 3)])
def test_hmc_moves_match_oracle(torch_cuda, N, n_sub, moves):
    from paper_1306_1821_gb300 import bps
    pb = Problem(N, n_sub=n_sub, n_bins=4, n_leapfrog=6, eps_max=0.4)
    s = pb.gpu(seed=21)
    try:
        ch = pb.oracle_chain(seed=21)
        for it in range(moves):
            acc, dH, eps = bps.bps_hmc_step(s.ctx)
            info = ch.hmc_step()
            ch.iteration += 1
            assert eps == pytest.approx(info["eps"], rel=1e-15)
            assert abs(dH - info["dH"]) < 1e-3, (dH, info["dH"])
            margin = abs(info["dH"] + math.log(info["u_acc"]))
            if margin > 1e-3:
                assert bool(acc) == info["accepted"]
            else:
                pytest.skip("decision within the tolerance band; states may legitimately differ")
            assert rel_l2(gpu_spectrum(s), ch.delta_hat) < 2e-4
    finally:
        s.close()


def test_hmc_accepts_and_moves(torch_cuda):
    # after a short burn-in from the (off-equilibrium) start, most moves are accepted
    from paper_1306_1821_gb300 import bps
    pb = Problem(32, n_sub=1, n_bins=4, n_leapfrog=8, eps_max=0.12)
    s = pb.gpu(seed=5)
    try:
        for _ in range(15):
            bps.bps_hmc_step(s.ctx)
        before = gpu_spectrum(s)
        acc = 0
        for _ in range(10):
            a, dH, eps = bps.bps_hmc_step(s.ctx)
            acc += a
            assert np.isfinite(dH) and 0 < eps < 0.12
        assert acc >= 5
        assert rel_l2(gpu_spectrum(s), before) > 1e-3
    finally:
        s.close()


@pytest.mark.parametrize("N,n_bins", [(16, 4), (32, 16), (64, 32)])
def test_power_sigma_and_draw(torch_cuda, N, n_bins):
    from paper_1306_1821_gb300 import bps
    pb = Problem(N, n_sub=1, n_bins=n_bins)
    s = pb.gpu(seed=9, iteration=4)
    try:
        P, sigma = bps.bps_sample_power(s.ctx, n_bins)
        ref_sigma = gibbs.bin_power(pb.geom, pb.dh)
        assert np.max(np.abs(sigma / ref_sigma - 1.0)) < 2e-6
        refP, _ = gibbs.sample_power(pb.geom, pb.dh, pb.wl.alpha, 9, 4)
        assert np.max(np.abs(P / refP - 1.0)) < 1e-5
    finally:
        s.close()


@pytest.mark.parametrize("N,n_sub", [(16, 2), (32, 3)])
def test_bias_norm_draw(torch_cuda, N, n_sub):
    from paper_1306_1821_gb300 import bps
    pb = Problem(N, n_sub=n_sub, n_bins=4)
    s = pb.gpu(seed=13, iteration=2)
    try:
        b, nbar, sums = bps.bps_sample_bias_norm(s.ctx, n_sub)
        delta = grid.inverse(pb.dh, N)
        ref_sums = gibbs.subsample_sums(delta, pb.counts, pb.R)
        scale = np.stack([np.sum(pb.counts[l] * np.abs(delta)) + np.sum(pb.R[l] * np.abs(delta)) +
                          np.sum(pb.R[l] * delta ** 2) for l in range(n_sub)])
        assert np.all(np.abs(sums - ref_sums) <= 1e-5 * scale[:, None])
        consts = gibbs.data_constants(pb.counts, pb.R)
        rb, rn = gibbs.sample_bias_norm(delta, ref_sums, consts, pb.b, pb.nbar, pb.wl.fixed_bias, 13, 2)
        for l in range(n_sub):
            C = pb.nbar[l] * ref_sums[l, 2]
            assert abs(b[l] - rb[l]) < 1e-3 / math.sqrt(C)
            assert nbar[l] == pytest.approx(rn[l], rel=1e-4)
        assert b[pb.wl.fixed_bias] == pb.b[pb.wl.fixed_bias]
    finally:
        s.close()


def test_jump_matches_oracle(torch_cuda):
    from paper_1306_1821_gb300 import bps
    pb = Problem(16, n_sub=1, n_bins=3, jump_leapfrog=4, jump_eps_max=0.3)
    s = pb.gpu(seed=17, iteration=1)
    try:
        ch = pb.oracle_chain(seed=17, iteration=1)
        for _ in range(3):
            acc, dH, eps = bps.bps_jump(s.ctx)
            info = ch.jump_step()
            ch.iteration += 1
            assert eps == pytest.approx(info["eps"], rel=1e-15)
            assert abs(dH - info["dH"]) < 1e-3
            assert bool(acc) == info["accepted"]
            P, _, _, _ = bps.bps_get_state(s.ctx, None, 3, 1)
            assert np.max(np.abs(P[:3] / ch.P - 1.0)) < 1e-5
            assert rel_l2(gpu_spectrum(s), ch.delta_hat) < 1e-5
    finally:
        s.close()


def test_gibbs_iterations_match_oracle(torch_cuda):
    from paper_1306_1821_gb300 import bps
    pb = Problem(16, n_sub=2, n_bins=3, n_leapfrog=5, eps_max=0.3, jump_leapfrog=3, jump_eps_max=0.2)
    s = pb.gpu(seed=23, jump=1)
    try:
        ch = pb.oracle_chain(seed=23, jump=True)
        n = 3
        rec = bps.bps_gibbs_iterate(s.ctx, n, s.rec_len)
        for i in range(n):
            r = ch.iterate()
            nb, ns = pb.wl.n_bins, pb.wl.n_sub
            assert np.max(np.abs(rec[i, :nb] / r["P"] - 1)) < 1e-4
            assert np.max(np.abs(rec[i, nb:nb + ns] - r["b"])) < 1e-3
            assert np.max(np.abs(rec[i, nb + ns:nb + 2 * ns] / r["nbar"] - 1)) < 1e-4
            assert abs(rec[i, -2] - r["hmc"]["dH"]) < 1e-3
        _, _, _, it = bps.bps_get_state(s.ctx, None, 3, 2)
        assert it == n
    finally:
        s.close()


def test_invalid_inputs_are_rejected(torch_cuda):
    from paper_1306_1821_gb300 import bps
    torch = torch_cuda
    with pytest.raises(bps.BpsError) as e:
        bps.bps_create(20, 100.0, 1, bps.make_config(2))
    assert e.value.status == bps.BPS_EINVAL
    with pytest.raises(bps.BpsError) as e:
        bps.bps_create(16, 100.0, 1, bps.make_config(16))   # first bin empty
    assert e.value.status == bps.BPS_EINVAL
    s = bps.Sampler(8, 100.0, 1, 2)
    try:
        with pytest.raises(bps.BpsError) as e:
            bps.bps_hmc_step(s.ctx)
        assert e.value.status == bps.BPS_ESTATE
        cnt = torch.zeros((1, 8, 8, 8), dtype=torch.int32, device="cuda")
        R = torch.ones((1, 8, 8, 8), dtype=torch.float32, device="cuda")
        R[0, 1, 1, 1] = -1.0
        with pytest.raises(bps.BpsError) as e:
            bps.bps_set_data(s.ctx, cnt, R)
        assert e.value.status == bps.BPS_EINVAL
        R[0, 1, 1, 1] = 0.0
        cnt[0, 1, 1, 1] = 3                                   # galaxies where R = 0
        with pytest.raises(bps.BpsError) as e:
            bps.bps_set_data(s.ctx, cnt, R)
        assert e.value.status == bps.BPS_EINVAL
        cnt[0, 1, 1, 1] = 0
        bps.bps_set_data(s.ctx, cnt, R)
        with pytest.raises(bps.BpsError):
            bps.bps_set_state(s.ctx, None, [-1.0, 1.0], [1.0], [1.0])
    finally:
        s.close()


def test_host_upload_equals_device_upload(torch_cuda):
    # the host path stages subsamples through two device slots on a copy stream
    from paper_1306_1821_gb300 import bps
    torch = torch_cuda
    pb = Problem(32, n_sub=3, n_bins=4, n_leapfrog=4, eps_max=0.2)
    a = pb.gpu(seed=13, jump=1)
    b = pb.gpu(seed=13, jump=1)
    try:
        bps.bps_set_data_host(b.ctx, np.ascontiguousarray(pb.counts), np.ascontiguousarray(pb.R))
        pinned_c = torch.from_numpy(pb.counts).pin_memory().numpy()
        pinned_r = torch.from_numpy(pb.R).pin_memory().numpy()
        bps.bps_set_data_host(b.ctx, pinned_c, pinned_r)        # twice: the slots are reused
        ra = bps.bps_gibbs_iterate(a.ctx, 2, a.rec_len)
        rb = bps.bps_gibbs_iterate(b.ctx, 2, b.rec_len)
        assert np.array_equal(ra, rb)
        # 16-bit counts from the host: the same data, the same chain
        c = pb.gpu(seed=13, jump=1)
        try:
            bps.bps_set_data_host_u16(c.ctx, pb.counts.astype(np.uint16), pb.R)
            rc = bps.bps_gibbs_iterate(c.ctx, 2, c.rec_len)
            assert np.array_equal(ra, rc)
        finally:
            c.close()
        bad = pb.counts.copy()
        bad[2, 0, 0, 0] = -1
        with pytest.raises(bps.BpsError):
            bps.bps_set_data_host(b.ctx, bad, pb.R)
    finally:
        a.close()
        b.close()


def test_tile_autotuner_choice_and_cache(torch_cuda, tmp_path, monkeypatch):
    # in a fresh process (the choice is cached per process): a new kind of
    # context times the tile sizes, keeps one and writes it to the cache file
    import json
    import os
    import subprocess
    import sys

    from paper_1306_1821_gb300 import bps
    path = tmp_path / "tune.json"
    code = ("from paper_1306_1821_gb300 import bps\n"
            "cfg = bps.make_config(2, n_leapfrog=2, eps_max=0.1)\n"
            "b = bps.bps_create_batch([8, 8, 8], [100.0] * 3, [1, 1, 1], cfg)\n"
            "print(bps.bps_x_pass_variant(b))\n"
            "print(bps.bps_z_line_pairs(b))\n"
            "bps.bps_destroy(b)\n")
    env = dict(os.environ, BPS_TUNE_CACHE=str(path))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lp = int(out.stdout.strip().splitlines()[-1])
    xv = int(out.stdout.strip().splitlines()[-2])
    assert lp in (4, 8, 16)
    assert xv in (0, 1, 2, 3, 4, 5, 6)
    cache = json.loads(path.read_text())
    assert any(k.endswith("N=8 chains=3 zpairs") and v == lp for k, v in cache.items())
    # the x-pass implementation (four with bit-identical results) is tuned and cached too
    assert any(k.endswith("N=8 chains=3 xleap") and v == xv for k, v in cache.items())
    monkeypatch.setenv("BPS_AUTOTUNE", "0")
    s = bps.Sampler(8, 100.0, 1, 2)
    try:
        assert bps.bps_z_line_pairs(s.ctx) == 8
        assert bps.bps_x_pass_variant(s.ctx) == 0
    finally:
        s.close()


def test_step_size_adaptation_moves_acceptance_toward_target(torch_cuda):
    from paper_1306_1821_gb300 import bps
    pb = Problem(16, n_sub=1, n_bins=4, n_leapfrog=6, eps_max=0.8)      # far too large a step
    s = pb.gpu(seed=5)
    try:
        def rate(n=40):
            acc = sum(bps.bps_hmc_step(s.ctx)[0] for _ in range(n))
            return acc / n
        before = rate()
        eps = bps.bps_adapt_step_size(s.ctx, 12, 20, 0.8)
        after = rate()
        assert eps < 0.8
        assert after > before
        assert abs(after - 0.8) < 0.2, (before, after, eps)
        with pytest.raises(bps.BpsError):
            bps.bps_adapt_step_size(s.ctx, 1, 1, 1.5)
    finally:
        s.close()


@pytest.mark.parametrize("fused", ["0", "1"])
def test_line_supports_at_the_ends_of_the_lines(torch_cuda, monkeypatch, fused):
    """Supports are rounded to multiples of four voxels: single observed voxels at
    z = 0 and z = N - 1, a fully observed line, a short run in the middle of a
    line and observed voxels in only one of two subsamples must all reach the force
    and the likelihood energy (three passes and the fused plane kernel)."""
    from paper_1306_1821_gb300 import bps
    monkeypatch.setenv("BPS_FUSED_YZ", fused)
    torch = torch_cuda
    N = 32
    pb = Problem(N, n_sub=2, n_bins=4)
    R = np.zeros_like(pb.R)
    counts = np.zeros_like(pb.counts)
    spots = [(0, 3, 5, 0), (0, 3, 6, N - 1), (1, 10, 1, 0), (1, 10, 1, N - 1), (0, 20, 20, 13),
             (1, 31, 0, 17), (0, 31, 31, N - 1)]
    for l, x, y, z in spots:
        R[l, x, y, z] = 0.8
        counts[l, x, y, z] = 2
    R[0, 7, 7, :] = 0.5                         # a fully observed line
    counts[0, 7, 7, ::3] = 1
    R[1, 12, 4, 9:14] = 1.2                     # a run inside one line
    counts[1, 12, 4, 10] = 4
    s = bps.Sampler(N, pb.wl.box, 2, pb.wl.n_bins, **pb.config_kwargs(11))
    try:
        bps.bps_set_data(s.ctx, torch.from_numpy(counts).cuda(), torch.from_numpy(R).cuda())
        bps.bps_set_state(s.ctx, None, pb.P, pb.b, pb.nbar, 0)
        bps.bps_set_spectrum(s.ctx, torch.from_numpy(pb.dh32).cuda())
        g = torch.zeros((N, N, N // 2 + 1), dtype=torch.complex64, device="cuda")
        e = bps.bps_gradient(s.ctx, g)
        a, c = model.local_fields(counts, R, pb.b, pb.nbar)
        gh, lik = model.gradient_hat(pb.geom, pb.dh, pb.P, a, c)
        assert rel_l2(g.cpu().numpy(), gh) < 1e-5
        assert abs(e[1] - lik) < 1e-5 * (abs(lik) + np.sum(np.abs(a * grid.inverse(pb.dh, N) ** 2)))
    finally:
        s.close()
