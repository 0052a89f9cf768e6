"""The leapfrog x pass with tensor-copy staged tiles (BPS_XTMA = 1, 2, 3) or a
ring of quarter tiles filled by tensor copies, by every thread's 16-byte copies or
by each warp for its own rows (BPS_XTMA = 4, 5, 6)
does the arithmetic of the direct-load pass in the same order, so its chains
must be bit-identical to the default's; and one of its HMC moves is checked
against the FP64 oracle (Sec. 4.1, the tolerances of tests/test_gpu_parity.py)."""
import math
import os

import numpy as np
import pytest

from tests.helpers import Problem, gpu_spectrum, rel_l2

pytestmark = pytest.mark.gpu


def chain(pb, variant, n_iter=2):
    old = os.environ.get("BPS_XTMA")
    os.environ["BPS_XTMA"] = str(variant)
    try:
        s = pb.gpu(seed=13, jump=1)
    finally:
        if old is None:
            del os.environ["BPS_XTMA"]
        else:
            os.environ["BPS_XTMA"] = old
    try:
        from paper_1306_1821_gb300 import bps
        rec = bps.bps_gibbs_iterate(s.ctx, n_iter, s.rec_len)
        return rec, gpu_spectrum(s)
    finally:
        s.close()


@pytest.mark.parametrize("N", [8, 16, 96, 256])
def test_staged_x_pass_equals_the_direct_pass(N):
    pb = Problem(N, n_sub=2, n_bins=3 if N == 8 else 8 if N < 256 else 32, n_leapfrog=4, eps_max=0.1 if N < 256 else 0.02)
    rec0, spec0 = chain(pb, 0)
    for v in (1, 2, 3, 4, 5, 6):
        rec, spec = chain(pb, v)
        assert np.array_equal(rec, rec0), v
        assert np.array_equal(spec, spec0), v


@pytest.mark.parametrize("variant", [1, 4, 5, 6])
def test_staged_x_pass_hmc_move_matches_oracle(variant):
    from paper_1306_1821_gb300 import bps
    pb = Problem(32, n_sub=2, n_bins=6, n_leapfrog=6, eps_max=0.25)
    os.environ["BPS_XTMA"] = str(variant)
    try:
        s = pb.gpu(seed=7)
    finally:
        del os.environ["BPS_XTMA"]
    try:
        acc, dH, eps = bps.bps_hmc_step(s.ctx)
        ch = pb.oracle_chain(seed=7)
        info = ch.hmc_step()
        assert abs(dH - info["dH"]) < 1e-3
        if abs(info["dH"] + math.log(info["u_acc"])) > 1e-3:
            assert bool(acc) == info["accepted"]
            assert rel_l2(gpu_spectrum(s), ch.delta_hat) < 2e-4
    finally:
        s.close()
