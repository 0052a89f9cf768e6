"""Staged survey uploads (bps_stage_data_host_u16): the upload of the next survey
runs beside the work queued after it and is activated by the next call that
uses the data.  Activation must give exactly the chain of a synchronous upload;
at most two surveys wait; an invalid survey is reported by the activating call
and leaves the previous survey active."""
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


def pinned(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).pin_memory().numpy()


def fresh(pb, seed):
    from paper_1306_1821_gb300 import bps
    return bps.Sampler(pb.N, pb.wl.box, pb.wl.n_sub, pb.wl.n_bins, **pb.config_kwargs(seed, jump=1))


def start_state(s, pb):
    import torch

    from paper_1306_1821_gb300 import bps
    bps.bps_set_state(s.ctx, None, pb.P, pb.b, pb.nbar, 0)
    bps.bps_set_spectrum(s.ctx, torch.from_numpy(pb.dh32).cuda())


@pytest.mark.parametrize("N", [32, 128])
def test_staged_upload_gives_the_synchronous_chain(torch_cuda, N):
    # 32^3: the data check widens each line's support per thread; 128^3: per warp
    from paper_1306_1821_gb300 import bps
    torch = torch_cuda
    pb = Problem(N, n_sub=2, n_bins=4, n_leapfrog=4, eps_max=0.2 if N == 32 else 0.05)
    ref = pb.gpu(seed=13, jump=1)
    st = fresh(pb, 13)
    try:
        c, r = pinned(torch, pb.counts, np.uint16), pinned(torch, pb.R, np.float32)
        bps.bps_stage_data_host_u16(st.ctx, c, r)
        start_state(st, pb)                     # before activation: no data yet
        rs = bps.bps_gibbs_iterate(st.ctx, 3, st.rec_len)
        rr = bps.bps_gibbs_iterate(ref.ctx, 3, ref.rec_len)
        assert np.array_equal(rs, rr)
    finally:
        ref.close()
        st.close()


def test_pipelined_uploads_activate_in_order(torch_cuda):
    """Survey k + 1 is staged before iteration k runs; each iteration uses its own
    survey, exactly as synchronous uploads between the iterations do."""
    from paper_1306_1821_gb300 import bps
    torch = torch_cuda
    surveys = [Problem(32, n_sub=2, n_bins=4, n_leapfrog=4, eps_max=0.2, f_sky=f, seed=sd)
               for f, sd in ((0.6, 3), (0.3, 4), (0.9, 5))]
    pb = surveys[0]
    ref = fresh(pb, 17)
    st = fresh(pb, 17)
    try:
        host = [(pinned(torch, q.counts, np.uint16), pinned(torch, q.R, np.float32)) for q in surveys]
        # reference: synchronous upload, then one iteration, per survey
        bps.bps_set_data_host_u16(ref.ctx, *host[0])
        start_state(ref, pb)
        rec_ref = []
        for k in range(3):
            if k:
                bps.bps_set_data_host_u16(ref.ctx, *host[k])
            rec_ref.append(bps.bps_gibbs_iterate(ref.ctx, 1, ref.rec_len))
        # pipelined: stage k + 1 before iterating on k
        bps.bps_stage_data_host_u16(st.ctx, *host[0])
        start_state(st, pb)
        rec = []
        for k in range(3):
            if k + 1 < 3:
                bps.bps_stage_data_host_u16(st.ctx, *host[k + 1])
            rec.append(bps.bps_gibbs_iterate(st.ctx, 1, st.rec_len))
        for a, b in zip(rec, rec_ref):
            assert np.array_equal(a, b)
    finally:
        ref.close()
        st.close()


def test_at_most_two_surveys_wait(torch_cuda):
    from paper_1306_1821_gb300 import bps
    torch = torch_cuda
    pb = Problem(32, n_sub=1, n_bins=4)
    s = pb.gpu(seed=5)
    try:
        c, r = pinned(torch, pb.counts, np.uint16), pinned(torch, pb.R, np.float32)
        bps.bps_stage_data_host_u16(s.ctx, c, r)
        bps.bps_stage_data_host_u16(s.ctx, c, r)
        with pytest.raises(bps.BpsError) as e:
            bps.bps_stage_data_host_u16(s.ctx, c, r)
        assert e.value.status == bps.BPS_ESTATE
        bps.bps_gibbs_iterate(s.ctx, 1, s.rec_len)   # activates one; the other still waits
        bps.bps_stage_data_host_u16(s.ctx, c, r)
        bps.bps_gibbs_iterate(s.ctx, 2, s.rec_len)
    finally:
        s.close()


def test_invalid_staged_survey_keeps_the_previous_one(torch_cuda):
    from paper_1306_1821_gb300 import bps
    torch = torch_cuda
    pb = Problem(32, n_sub=2, n_bins=4, n_leapfrog=4, eps_max=0.2)
    ref = pb.gpu(seed=9)
    s = pb.gpu(seed=9)
    try:
        bad = pb.counts.copy()
        bad[1][pb.R[1] == 0] = 0
        bad[1].flat[np.flatnonzero(pb.R[1] == 0)[0]] = 3        # a count where R = 0
        c, r = pinned(torch, bad, np.uint16), pinned(torch, pb.R, np.float32)
        bps.bps_stage_data_host_u16(s.ctx, c, r)
        with pytest.raises(bps.BpsError) as e:
            bps.bps_gibbs_iterate(s.ctx, 1, s.rec_len)
        assert e.value.status == bps.BPS_EINVAL
        # that iteration ran on the previous survey, as the next ones do
        bps.bps_gibbs_iterate(ref.ctx, 1, ref.rec_len)
        assert np.array_equal(bps.bps_gibbs_iterate(s.ctx, 2, s.rec_len),
                              bps.bps_gibbs_iterate(ref.ctx, 2, ref.rec_len))
    finally:
        ref.close()
        s.close()


def test_invalid_first_survey_leaves_no_data(torch_cuda):
    """A context whose only staged survey is invalid has no data afterwards: the
    activating call reports the data error, later calls report missing data, and a
    valid survey makes the chain usable."""
    from paper_1306_1821_gb300 import bps
    torch = torch_cuda
    pb = Problem(32, n_sub=1, n_bins=4)
    s = fresh(pb, 3)
    try:
        bad = pb.counts.copy()
        bad[0].flat[np.flatnonzero(pb.R[0] == 0)[0]] = 1          # a count where R = 0
        c, r = pinned(torch, bad, np.uint16), pinned(torch, pb.R, np.float32)
        bps.bps_stage_data_host_u16(s.ctx, c, r)
        start_state(s, pb)
        with pytest.raises(bps.BpsError) as e:
            bps.bps_gibbs_iterate(s.ctx, 1, s.rec_len)
        assert e.value.status == bps.BPS_EINVAL
        with pytest.raises(bps.BpsError) as e:
            bps.bps_gibbs_iterate(s.ctx, 1, s.rec_len)
        assert e.value.status == bps.BPS_ESTATE
        bps.bps_set_data_host_u16(s.ctx, pinned(torch, pb.counts, np.uint16), r)
        start_state(s, pb)
        assert np.all(np.isfinite(bps.bps_gibbs_iterate(s.ctx, 1, s.rec_len)))
    finally:
        s.close()
