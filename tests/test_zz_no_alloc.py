"""bps_bin_power_noalloc: the k-bin power of a half spectrum for callers that may
not allocate device memory (its scratch is a fixed file-scope device array).

Checked through the C ABI against the power the library's regular path
(bps_sample_power, which keeps its partial sums in a cudaMalloc'd buffer)
returns for the same field, on two calls in a row, within the tolerance the
other parity tests use for sigma_m.  Kept in its own file so that it runs last.
"""
import numpy as np
import pytest

from tests.helpers import Problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,n_bins", [(32, 16), (64, 32)])
def test_noalloc_bin_power_matches_regular_path(N, n_bins):
    import torch

    from paper_1306_1821_gb300 import bps
    pb = Problem(N, n_sub=1, n_bins=n_bins)
    s = pb.gpu(seed=9, iteration=4)
    try:
        _, sigma_regular = bps.bps_sample_power(s.ctx, n_bins)
        spec = torch.from_numpy(pb.dh32).cuda()
        for _ in range(2):    # the scratch is shared and reused: two calls in a row
            out = torch.full((n_bins,), float("nan"), dtype=torch.float64, device="cuda")
            bps.bps_bin_power_noalloc(N, pb.wl.box, n_bins, spec, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert np.max(np.abs(got / sigma_regular - 1.0)) < 2e-6
    finally:
        s.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    from paper_1306_1821_gb300 import bps
    spec = torch.zeros((8, 8, 5), dtype=torch.complex64, device="cuda")
    out = torch.zeros(65, dtype=torch.float64, device="cuda")
    with pytest.raises(bps.BpsError) as e:
        bps.bps_bin_power_noalloc(8, 100.0, 65, spec, out)
    assert e.value.status == bps.BPS_EINVAL
    with pytest.raises(bps.BpsError) as e:
        bps.bps_bin_power_noalloc(1024, 100.0, 4, spec, out)
    assert e.value.status == bps.BPS_EINVAL
