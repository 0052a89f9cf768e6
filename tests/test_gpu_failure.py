"""Failure detection and checkpoint/resume through the C ABI, in forms that
fault, trap or hang nothing.

  * A bounded device wait that runs out: bps_selftest_wait waits on an
    mbarrier that no copy completes (none is issued), with a short limit; the
    call must return BPS_ETIMEOUT and the context must stay usable.
  * A non-finite state: a half spectrum with a NaN mode, injected from the
    host.  The HMC move's energy difference is not finite, the Metropolis step
    (Eq. acceptance_rule) must reject it and the call return BPS_ENUMERIC with
    the chain's state untouched; a finite state set afterwards moves again.
  * Resume: a checkpoint (bps_save_chain) loaded into a fresh context holding
    the same survey continues the chain bit for bit, with the jump on; and the
    plain state calls (bps_get_state / bps_set_state, the spectrum) do the same
    for a chain without the jump (whose reference spectrum is unused).
"""
import numpy as np
import pytest

from tests.helpers import Problem, gpu_spectrum

pytestmark = pytest.mark.gpu


def _copy_of(pb, seed, jump):
    """A fresh context with the same settings and survey as pb.gpu(), no state."""
    import torch

    from paper_1306_1821_gb300 import bps
    s = bps.Sampler(pb.N, pb.wl.box, pb.wl.n_sub, pb.wl.n_bins, **pb.config_kwargs(seed, jump))
    bps.bps_set_data(s.ctx, torch.from_numpy(pb.counts).cuda(), torch.from_numpy(pb.R).cuda())
    return s


def test_wait_timeout_is_reported_and_the_context_stays_usable():
    from paper_1306_1821_gb300 import bps
    pb = Problem(16, n_sub=1, n_bins=4)
    s = pb.gpu(seed=3)
    try:
        before = gpu_spectrum(s)
        with pytest.raises(bps.BpsError) as e:
            bps.bps_selftest_wait(s.ctx, 20000)        # 20 microseconds
        assert e.value.status == bps.BPS_ETIMEOUT
        assert "wait limit" in str(e.value)
        assert np.array_equal(gpu_spectrum(s), before)
        acc, dH, eps = bps.bps_hmc_step(s.ctx)          # the context still works
        assert np.isfinite(dH)
        with pytest.raises(bps.BpsError) as e:
            bps.bps_selftest_wait(s.ctx, 0)
        assert e.value.status == bps.BPS_EINVAL
    finally:
        s.close()


def test_non_finite_state_is_rejected_and_kept():
    import torch

    from paper_1306_1821_gb300 import bps
    pb = Problem(32, n_sub=2, n_bins=8)
    s = pb.gpu(seed=5)
    try:
        bad = pb.dh32.copy()
        bad[3, 5, 7] = np.complex64(np.nan)
        bps.bps_set_spectrum(s.ctx, torch.from_numpy(bad).cuda())
        with pytest.raises(bps.BpsError) as e:
            bps.bps_hmc_step(s.ctx)
        assert e.value.status == bps.BPS_ENUMERIC
        assert "non-finite" in str(e.value)
        raw = torch.zeros((32, 32, 17), dtype=torch.complex64, device="cuda")
        bps.bps_get_spectrum(s.ctx, raw)
        got = raw.cpu().numpy()
        assert np.array_equal(got.view(np.uint64), bad.view(np.uint64))   # NaN bits included
        bps.bps_set_spectrum(s.ctx, torch.from_numpy(pb.dh32).cuda())
        acc, dH, eps = bps.bps_hmc_step(s.ctx)
        assert np.isfinite(dH)
    finally:
        s.close()


def test_checkpoint_resume_continues_the_chain_bit_for_bit():
    from paper_1306_1821_gb300 import bps
    pb = Problem(32, n_sub=2, n_bins=8, n_leapfrog=5, eps_max=0.2, jump_leapfrog=4, jump_eps_max=0.3)
    a = pb.gpu(seed=21, jump=1)
    b = _copy_of(pb, seed=21, jump=1)
    try:
        bps.bps_gibbs_iterate(a.ctx, 3, a.rec_len)
        blob = bps.bps_save_chain(a.ctx)
        rec_a = bps.bps_gibbs_iterate(a.ctx, 4, a.rec_len)
        bps.bps_load_chain(b.ctx, blob)
        rec_b = bps.bps_gibbs_iterate(b.ctx, 4, b.rec_len)
        assert np.array_equal(rec_a, rec_b)
        assert np.array_equal(gpu_spectrum(a), gpu_spectrum(b))
        assert bps.bps_get_state(a.ctx, None, 8, 2)[3] == bps.bps_get_state(b.ctx, None, 8, 2)[3]
        # a checkpoint of another grid is refused
        c = Problem(16, n_sub=2, n_bins=8).gpu(seed=21, jump=1)
        try:
            with pytest.raises(bps.BpsError) as e:
                bps.bps_load_chain(c.ctx, blob)
            assert e.value.status == bps.BPS_EINVAL
            with pytest.raises(bps.BpsError) as e:
                bps.bps_load_chain(c.ctx, blob[:100])
            assert e.value.status == bps.BPS_EINVAL
        finally:
            c.close()
    finally:
        a.close()
        b.close()


def test_state_calls_resume_a_chain_without_the_jump():
    import torch

    from paper_1306_1821_gb300 import bps
    pb = Problem(32, n_sub=2, n_bins=8, n_leapfrog=5, eps_max=0.2)
    a = pb.gpu(seed=23, jump=0)
    b = _copy_of(pb, seed=23, jump=0)
    try:
        bps.bps_gibbs_iterate(a.ctx, 2, a.rec_len)
        P, bb, nb, it = bps.bps_get_state(a.ctx, None, 8, 2)
        spec = torch.zeros((32, 32, 17), dtype=torch.complex64, device="cuda")
        bps.bps_get_spectrum(a.ctx, spec)
        rec_a = bps.bps_gibbs_iterate(a.ctx, 3, a.rec_len)
        bps.bps_set_state(b.ctx, None, P, bb[:2], nb[:2], it)
        bps.bps_set_spectrum(b.ctx, spec)
        rec_b = bps.bps_gibbs_iterate(b.ctx, 3, b.rec_len)
        assert np.array_equal(rec_a, rec_b)
    finally:
        a.close()
        b.close()
