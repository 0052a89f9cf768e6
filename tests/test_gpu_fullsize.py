"""Parity at the benchmark's full size: the 256^3 six-subsample survey with 32
k bins, in the launch configuration bench.py times (single context, the same
kernels and tile choices).  One HMC move against the FP64 oracle and the k-bin
power of the resulting field.

Delta H tolerance at this size.  The fields are FP32: a transform of N^3 points
leaves a relative error of about u sqrt(log2 N^3) ~ 3e-7 per voxel (unit
roundoff u = 6e-8), and the likelihood energy weighs each voxel's delta by the
local drive 2 c (a few units with six subsamples), so each energy carries a
random error of order sqrt(N^3) * 2 c * 3e-7 * |delta| ~ 1e-2 at 256^3.  The
errors of H0 and H1 are largely correlated and the difference keeps a part of
it: measured |Delta H - Delta H_oracle| = 1.9e-3 (and 2e-3 to 4e-3 at
|Delta H| ~ 30).  The test allows 5e-3; at the parity-test sizes (16^3-128^3)
the 1e-3 bound holds and is tested there.  The Metropolis decision must agree
unless |Delta H + ln u| is within that band."""
import math
from dataclasses import replace

import numpy as np
import pytest

from oracle import gibbs
from paper_1306_1821_gb300 import inputs
from tests.helpers import Problem, gpu_spectrum, rel_l2

pytestmark = pytest.mark.gpu


def test_hmc_move_and_bin_power_at_256():
    from paper_1306_1821_gb300 import bps
    wl = replace(inputs.WORKLOADS["survey256"], n_leapfrog=4, eps_max=0.02, jump=False)   # |dH| of order 1
    pb = Problem(256, wl=wl)
    s = pb.gpu(seed=3)
    try:
        acc, dH, eps = bps.bps_hmc_step(s.ctx)
        ch = pb.oracle_chain(seed=3)
        info = ch.hmc_step()
        assert eps == pytest.approx(info["eps"], rel=1e-15)
        assert abs(dH - info["dH"]) < 5e-3, (dH, info["dH"])
        if abs(info["dH"] + math.log(info["u_acc"])) > 5e-3:
            assert bool(acc) == info["accepted"]
            assert rel_l2(gpu_spectrum(s), ch.delta_hat) < 2e-4
        P, sigma = bps.bps_sample_power(s.ctx, wl.n_bins)
        ref = gibbs.bin_power(pb.geom, gpu_spectrum(s))
        assert np.max(np.abs(sigma / ref - 1)) < 2e-6
    finally:
        s.close()
