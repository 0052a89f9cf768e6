"""Parity at the library's limits: 64 power-spectrum bins (MAXB, which needs
N >= 128 so that the first bin holds a mode) and 16 galaxy subsamples (MAXS),
each against the FP64 oracle through the C ABI, and a Gibbs scan with both at
once.  Tolerances as in test_gpu_parity.py."""
import math
from dataclasses import replace

import numpy as np
import pytest

from oracle import gibbs, grid
from paper_1306_1821_gb300 import inputs
from tests.helpers import Problem, compare_chain

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    from paper_1306_1821_gb300 import bps
    bps.load()
    return torch


def limit_workload(N, n_sub, n_bins, **kw):
    """The small-workload recipe with n_sub subsamples: biases 1.0 .. 1.75 and
    mean numbers 8 .. 0.5 per voxel (geometric), the first bias fixed."""
    base = inputs.small_workload(N, n_bins=n_bins, n_sub=1, **kw)
    b = [1.0 + 0.05 * l for l in range(n_sub)]
    nbar = [8.0 * (1.0 / 16.0) ** (l / max(n_sub - 1, 1)) for l in range(n_sub)]
    return replace(base, name=f"limits{N}", b=b, nbar=nbar)


def test_power_at_64_bins(torch_cuda):
    from paper_1306_1821_gb300 import bps
    pb = Problem(128, wl=limit_workload(128, 1, 64))
    s = pb.gpu(seed=9, iteration=4)
    try:
        P, sigma = bps.bps_sample_power(s.ctx, 64)
        ref_sigma = gibbs.bin_power(pb.geom, pb.dh)
        assert np.all(pb.geom.n_modes > 0)
        assert np.max(np.abs(sigma / ref_sigma - 1.0)) < 2e-6
        refP, _ = gibbs.sample_power(pb.geom, pb.dh, pb.wl.alpha, 9, 4)
        assert np.max(np.abs(P / refP - 1.0)) < 1e-5
    finally:
        s.close()


def test_bias_norm_draw_at_16_subsamples(torch_cuda):
    from paper_1306_1821_gb300 import bps
    n_sub = 16
    pb = Problem(32, wl=limit_workload(32, n_sub, 4, seed=5))
    s = pb.gpu(seed=13, iteration=2)
    try:
        b, nbar, sums = bps.bps_sample_bias_norm(s.ctx, n_sub)
        delta = grid.inverse(pb.dh, pb.N)
        ref_sums = gibbs.subsample_sums(delta, pb.counts, pb.R)
        scale = np.stack([np.sum(pb.counts[l] * np.abs(delta)) + np.sum(pb.R[l] * np.abs(delta)) +
                          np.sum(pb.R[l] * delta ** 2) for l in range(n_sub)])
        assert np.all(np.abs(sums - ref_sums) <= 1e-5 * scale[:, None])
        consts = gibbs.data_constants(pb.counts, pb.R)
        rb, rn = gibbs.sample_bias_norm(delta, ref_sums, consts, pb.b, pb.nbar, pb.wl.fixed_bias, 13, 2)
        for l in range(n_sub):
            C = pb.nbar[l] * ref_sums[l, 2]
            assert abs(b[l] - rb[l]) < 1e-3 / math.sqrt(C), l
            assert nbar[l] == pytest.approx(rn[l], rel=1e-4), l
        assert b[pb.wl.fixed_bias] == pb.b[pb.wl.fixed_bias]
    finally:
        s.close()


def test_gibbs_iterations_at_64_bins_and_16_subsamples(torch_cuda):
    from paper_1306_1821_gb300 import bps
    wl = limit_workload(128, 16, 64, n_leapfrog=3, eps_max=0.05, jump_leapfrog=2, jump_eps_max=0.1, seed=7)
    pb = Problem(128, wl=wl)
    s = pb.gpu(seed=29, jump=1)
    try:
        n = 2
        rec = bps.bps_gibbs_iterate(s.ctx, n, s.rec_len)
        assert rec.shape == (n, 64 + 2 * 16 + 2)
        ch = pb.oracle_chain(seed=29, jump=True)
        done, worst = compare_chain(rec, ch, n)
        print(f"limits: {done} iterations compared, max |dH - dH_oracle| = {worst:.2e}")
        assert done >= 1
    finally:
        s.close()
