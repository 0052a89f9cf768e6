"""Kernel timing (bps_profile / bps_profile_read) through the C ABI: timing
changes nothing in the chain, profiled iterations replay a captured iteration
with event-record nodes around the leapfrog kernels, and every leapfrog step
of every profiled iteration is counted once per kernel kind."""
import numpy as np
import pytest

from tests.helpers import Problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    from paper_1306_1821_gb300 import bps
    bps.load()
    return torch


@pytest.mark.parametrize("N", [32, 64])
def test_profiled_iterations_give_the_same_chain_and_count_every_step(torch_cuda, N):
    from paper_1306_1821_gb300 import bps
    L = 5
    pb = Problem(N, n_sub=2, n_bins=4, n_leapfrog=L, eps_max=0.2 if N == 32 else 0.1)
    ref = pb.gpu(seed=21, jump=1)
    prof = pb.gpu(seed=21, jump=1)
    try:
        rec_ref = bps.bps_gibbs_iterate(ref.ctx, 7, ref.rec_len)
        l_ref = bps.bps_kernel_launches(ref.ctx)
        # plain, profiled one at a time, profiled in a run of three
        recs = [bps.bps_gibbs_iterate(prof.ctx, 2, prof.rec_len)]
        bps.bps_profile(prof.ctx, 1)
        recs.append(bps.bps_gibbs_iterate(prof.ctx, 1, prof.rec_len))
        recs.append(bps.bps_gibbs_iterate(prof.ctx, 1, prof.rec_len))
        recs.append(bps.bps_gibbs_iterate(prof.ctx, 3, prof.rec_len))
        bps.bps_profile(prof.ctx, 0)
        ms, n = bps.bps_profile_read(prof.ctx)
        # the same kernels, plus one record reset per call
        assert bps.bps_kernel_launches(prof.ctx) == l_ref + 3
        # nothing is timed once timing is off
        bps.bps_gibbs_iterate(prof.ctx, 1, prof.rec_len)
        ms2, n2 = bps.bps_profile_read(prof.ctx)
    finally:
        ref.close()
        prof.close()
    rec = np.concatenate(recs, 0)
    assert np.array_equal(rec, rec_ref)
    profiled = 5
    assert n[0] == L * profiled and n[2] == L * profiled
    # kinds 1 and 3 (the y passes) exist when the force stage runs as three passes
    assert n[1] == n[3] and n[1] in (0, L * profiled)
    assert np.all(ms[n > 0] > 0) and np.all(ms[n > 0] / n[n > 0] < 10.0)
    assert np.all(n2 == 0) and np.all(ms2 == 0)
