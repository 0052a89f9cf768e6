"""bps_bin_power_noalloc: the k-bin power of a half spectrum for callers that may
not allocate device memory (its scratch is a fixed file-scope device array).

Checked through the C ABI element by element against the FP64 oracle's sigma_m
(oracle.gibbs.bin_power, Sec. 3.4) on caller spectra with a nonzero k = 0 mode
(which belongs to no bin and must be ignored), at grid sizes only this entry
point accepts (6, 48, 200), at 128 and 256 (more half-spectrum rows than the
fixed grid has warps, so every warp takes several rows), and at the 64-bin
limit; each on two calls in a row, since every call reuses the same scratch.
Tolerance 2e-6 relative: the terms are positive, FP32 per element, and summed
in FP64 from per-warp segments.  Also checked against the regular path
(bps_sample_power, whose partial sums live in a cudaMalloc'd buffer).  Kept in
its own file so that it runs last.
"""
import numpy as np
import pytest

from oracle import gibbs, grid
from tests.helpers import Problem

pytestmark = pytest.mark.gpu


def caller_spectrum(N, seed):
    """A complex64 half spectrum [N][N][N/2+1] with independent random modes,
    the k = 0 mode included (nonzero)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (N, N, N // 2 + 1)
    spec = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    spec[0, 0, 0] = 250.0 + 40.0j
    return spec


@pytest.mark.parametrize("N,n_bins", [(6, 3), (48, 24), (128, 64), (200, 64), (256, 32)])
def test_noalloc_bin_power_matches_oracle(N, n_bins):
    import torch

    from paper_1306_1821_gb300 import bps
    box = 7.0 * N
    spec = caller_spectrum(N, seed=N)
    ref = gibbs.bin_power(grid.Geometry(N, box, n_bins), spec.astype(np.complex128))
    assert np.all(ref > 0)
    dspec = torch.from_numpy(spec).cuda()
    for _ in range(2):
        out = torch.full((n_bins,), float("nan"), dtype=torch.float64, device="cuda")
        bps.bps_bin_power_noalloc(N, box, n_bins, dspec, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got / ref - 1.0)) < 2e-6, np.max(np.abs(got / ref - 1.0))


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
    for args in [(8, 100.0, 65), (1024, 100.0, 4), (7, 100.0, 2)]:
        with pytest.raises(bps.BpsError) as e:
            bps.bps_bin_power_noalloc(*args, spec, out)
        assert e.value.status == bps.BPS_EINVAL


def test_noalloc_rejects_empty_bins_and_misaligned_pointers():
    import torch

    from paper_1306_1821_gb300 import bps
    spec = torch.zeros((32, 32, 17), dtype=torch.complex64, device="cuda")
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    # 64 bins on a 32^3 grid: the first bin ends below |n| = 1 and holds no mode
    # (bps_create rejects the same layout)
    with pytest.raises(bps.BpsError) as e:
        bps.bps_bin_power_noalloc(32, 100.0, 64, spec, out)
    assert e.value.status == bps.BPS_EINVAL
    # a float view one element into the spectrum is 4-byte aligned only
    flat = torch.zeros(2 * 32 * 32 * 17 + 2, dtype=torch.float32, device="cuda")
    with pytest.raises(bps.BpsError) as e:
        bps.bps_bin_power_noalloc(32, 100.0, 8, flat[1:], out)
    assert e.value.status == bps.BPS_EINVAL
    # nothing was queued by the rejected calls; a valid call still works
    bps.bps_bin_power_noalloc(32, 100.0, 8, spec, out)
    torch.cuda.synchronize()
    assert np.all(out[:8].cpu().numpy() == 0.0)
