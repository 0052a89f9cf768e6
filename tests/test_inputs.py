"""The seeded input generator (paper_1306_1821_gb300/inputs.py) against the
recipe it states: a Gaussian field of voxel variance 0.5 with the given power
spectrum, a spherical-cap response times the radial selection, and Poisson
counts of mean R Nbar max(0, 1 + b delta) that vanish where R = 0."""
import math

import numpy as np

from paper_1306_1821_gb300 import inputs


def full_grid_k(N, box):
    n = np.fft.fftfreq(N, 1.0 / N)
    nx, ny, nz = np.meshgrid(n, n, n, indexing="ij")
    return 2.0 * np.pi * np.sqrt(nx * nx + ny * ny + nz * nz) / box


def test_amplitude_gives_the_stated_voxel_variance():
    # (1/V) sum of P(k) over every non-DC mode of the full grid = 0.5
    for N, box in [(16, 250.0), (32, 500.0), (48, 900.0)]:
        k = full_grid_k(N, box)
        P = inputs.true_spectrum(k[k > 0], N, box)
        assert math.isclose(np.sum(P) / box ** 3, 0.5, rel_tol=1e-12)


def test_field_power_counts_and_response_follow_the_recipe():
    wl = inputs.small_workload(32, n_sub=2, f_sky=0.4, seed=11)
    delta, counts, R = inputs.make_survey(wl)
    N, box = wl.N, wl.box
    # E |delta_hat_k|^2 = N_v P_k / V_cell: the mean ratio over ~16k half-spectrum modes is 1
    dh = np.fft.rfftn(delta)
    k = inputs.wavenumbers(N, box)
    ratio = np.abs(dh[k > 0]) ** 2 / (N ** 3 * inputs.true_spectrum(k[k > 0], N, box) / (box / N) ** 3)
    assert abs(ratio.mean() - 1.0) < 0.04
    # counts vanish where the response does, and their total is Poisson about its mean
    assert np.all(counts[R == 0] == 0)
    for l in range(wl.n_sub):
        lam = R[l].astype(np.float64) * wl.nbar[l] * np.maximum(0.0, 1.0 + wl.b[l] * delta)
        assert abs(counts[l].sum() - lam.sum()) < 5.0 * math.sqrt(lam.sum())
    # the response: zero beyond L/2, the cap covers f_sky of the sky in a thin shell
    c = (np.arange(N) + 0.5) * (box / N) - box / 2.0
    x, y, z = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    assert np.all(R[:, r > box / 2.0] == 0)
    shell = (r > 0.3 * box / 2.0) & (r < box / 2.0)
    assert abs(np.mean(R[0][shell] > 0) - wl.f_sky) < 0.03
    # same seed, same survey
    d2, c2, R2 = inputs.make_survey(wl)
    assert np.array_equal(d2, delta) and np.array_equal(c2, counts) and np.array_equal(R2, R)
