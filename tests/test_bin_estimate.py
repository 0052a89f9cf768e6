"""The field passes find the bin of |n|^2 from an FP32 estimate
floor(sqrt(n2) * nb / (sqrt(3) N / 2)) corrected by at most one bin against the
exact integer thresholds.  This checks, for every supported grid (and N = 512)
and every bin count 1..64, that the estimate computed with the device's FP32
operations is never more than one bin away from the exact FP64 bin."""
import numpy as np
import pytest

from oracle.grid import bin_of_n2


@pytest.mark.parametrize("N", [8, 16, 32, 64, 96, 128, 256, 512])
def test_fp32_bin_estimate_is_within_one_bin(N):
    n2 = np.arange(1, 3 * (N // 2) ** 2 + 1, dtype=np.int64)
    root = np.sqrt(n2.astype(np.float32))                       # sqrtf: correctly rounded
    for nb in range(1, 65):
        scale = np.float32(nb) / (np.float32(0.8660254) * np.float32(N))
        est = np.minimum(nb - 1, (root * scale).astype(np.int64))
        exact = bin_of_n2(n2, N, nb)
        assert np.abs(est - exact).max() <= 1, (N, nb)
