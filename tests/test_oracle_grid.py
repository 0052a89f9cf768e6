"""Pins of the oracle's Fourier convention (App. C.1) and k-binning."""
import numpy as np
import pytest

from oracle import grid


def naive_dft3(x, sign):
    """O(N^6) literal sum of Eq. FFT / Eq. IFFT (without normalisation)."""
    N = x.shape[0]
    j = np.arange(N)
    F = np.exp(sign * 2j * np.pi * np.outer(j, j) / N)
    out = np.einsum("ai,bj,ck,ijk->abc", F, F, F, x.astype(np.complex128))
    return out


@pytest.mark.parametrize("N", [4, 6, 8])
def test_forward_inverse_against_literal_dft(N):
    rng = np.random.default_rng(N)
    x = rng.standard_normal((N, N, N))
    full = naive_dft3(x, -1.0)                      # C_hat = 1
    half = grid.forward(x)
    assert np.allclose(half, full[:, :, : N // 2 + 1], atol=1e-10)
    back = grid.inverse(half, N)                   # C = 1 / N_vox
    lit = naive_dft3(full, +1.0).real / N ** 3
    assert np.allclose(back, lit, atol=1e-12)
    assert np.allclose(back, x, atol=1e-12)


@pytest.mark.parametrize("N", [4, 8, 12])
def test_half_spectrum_weights_reproduce_full_grid_sums(N):
    g = grid.Geometry(N, 100.0, 3)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((N, N, N))
    full = np.fft.fftn(x)
    half = grid.forward(x)
    assert np.sum(g.w * np.abs(half) ** 2) == pytest.approx(np.sum(np.abs(full) ** 2), rel=1e-12)
    # Parseval under App. C.1: sum_i x_i^2 = (1/N_vox) sum_k |x_hat_k|^2
    assert np.sum(x * x) == pytest.approx(np.sum(g.w * np.abs(half) ** 2) / N ** 3, rel=1e-12)


@pytest.mark.parametrize("N,nb", [(4, 1), (8, 5), (16, 8), (32, 16), (64, 32)])
def test_bins_partition_all_nonzero_modes(N, nb):
    g = grid.Geometry(N, 500.0, nb)
    assert g.bin[0, 0, 0] == -1
    assert np.sum(g.bin < 0) == 1
    assert g.n_modes.sum() == N ** 3 - 1
    assert np.all(g.n_modes > 0)
    # bin index is non-decreasing in |n|
    n2 = g.n2.ravel()
    b = g.bin.ravel()
    order = np.argsort(n2, kind="stable")
    assert np.all(np.diff(b[order][1:]) >= 0)
    # the corner mode sqrt(3) N / 2 lands in the last bin
    assert grid.bin_of_n2(3 * (N // 2) ** 2, N, nb) == nb - 1
    # full-grid count by brute force over all N^3 integer vectors
    i = np.arange(N)
    s = np.where(i <= N // 2, i, i - N)
    n2_full = (s[:, None, None] ** 2 + s[None, :, None] ** 2 + s[None, None, :] ** 2).ravel()
    bf = grid.bin_of_n2(n2_full, N, nb)
    counts = np.bincount(bf[bf >= 0], minlength=nb)
    assert np.array_equal(counts, g.n_modes.astype(int))


def test_too_many_bins_leave_the_first_bin_empty():
    # with n_bins = N the first bin spans |n| < sqrt(3)/2 and holds no mode; the
    # library rejects such a layout
    g = grid.Geometry(16, 500.0, 16)
    assert g.n_modes[0] == 0
