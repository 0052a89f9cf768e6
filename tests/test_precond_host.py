"""Host logic of the preconditioner harness (precond.py), without a GPU: the
random training problems, the radial table its device mocks use, the features,
the standardisation clamp and the network initialisation."""
import math
from dataclasses import replace

import numpy as np
import pytest

from oracle import mock
from paper_1306_1821_gb300 import inputs, precond


@pytest.mark.parametrize("radial", ["linear", "gauss"])
def test_radial_table_reproduces_the_inputs_response(radial):
    # cap x the table, linearly interpolated (the mock response's definition),
    # must give the host recipe's response voxel for voxel
    base = inputs.small_workload(32, f_sky=0.35)
    wl = replace(base, radial=radial, extra={"axis": (0.3, -0.2, 0.9)})
    table = precond.radial_table(wl)
    assert table.shape == (wl.n_sub, 2049)
    R_mock = mock.response(wl.N, wl.box, wl.f_sky, wl.extra["axis"], table, wl.box / 2.0)[0]
    R_host = inputs.response(wl.N, wl.box, wl.f_sky, radial, wl.r0, wl.extra["axis"])
    assert np.array_equal(R_mock > 0, R_host > 0)
    # a linear selection is interpolated exactly; a Gaussian one to the float32 rounding
    assert np.max(np.abs(R_mock - R_host)) <= (0.0 if radial == "linear" else 2.5e-7)


def test_random_problems_are_seeded_and_in_range():
    base = inputs.WORKLOADS["survey32"]
    ps = precond.random_problems(base, 6, 100)
    again = precond.random_problems(base, 6, 100)
    bc = inputs.bin_centre_spectrum(base.N, base.box, base.n_bins)
    for p, q in zip(ps, again):
        assert p.wl.f_sky == q.wl.f_sky and p.wl.extra == q.wl.extra and np.array_equal(p.P, q.P)
        assert 0.2 <= p.wl.f_sky <= 0.6
        assert math.isclose(np.linalg.norm(p.wl.extra["axis"]), 1.0, rel_tol=1e-12)
        lr = np.log(p.P / bc)
        assert np.all(lr > math.log(0.5) - 0.6) and np.all(lr < math.log(2.0) + 0.6)
        # grid, box, subsamples and radial selection are the base workload's
        assert (p.wl.N, p.wl.box, p.wl.b, p.wl.nbar, p.wl.radial) == (base.N, base.box, base.b, base.nbar, base.radial)
    assert len({p.wl.seed for p in ps}) == 6
    assert len({round(p.wl.f_sky, 12) for p in ps}) == 6


def test_features_standardisation_and_initialisation():
    P = np.array([2.0, 3.0])
    W = np.array([0.5, 0.0])
    f = precond.features(P, W)
    assert np.allclose(f, [math.log(2.0), math.log(3.0), math.log(0.5), math.log(1e-30)])
    # standardised features are clamped to +-4, as the library clamps them on the device
    p = precond.Preconditioner.__new__(precond.Preconditioner)
    p.mu = np.array([0.0, 1.0])
    p.sd = np.array([1.0, 0.5])
    z = p.standardise(np.array([[10.0, 1.25], [-0.5, -9.0]]))
    assert z.dtype == np.float32
    assert np.allclose(z, [[4.0, 0.5], [-0.5, -4.0]])
    # He-uniform weights within +-sqrt(6 / n_in), zero biases, seeded
    sizes = [32, 128, 128, 64]
    a, b = precond.he_init(sizes, 5), precond.he_init(sizes, 5)
    assert len(a) == 6
    for i, (n_in, n_out) in enumerate(zip(sizes[:-1], sizes[1:])):
        Wi, bi = a[2 * i], a[2 * i + 1]
        assert Wi.shape == (n_in, n_out) and np.all(bi == 0)
        assert np.max(np.abs(Wi)) <= math.sqrt(6.0 / n_in)
        assert abs(Wi.std() - math.sqrt(2.0 / n_in)) < 0.1 * math.sqrt(2.0 / n_in)
        assert np.array_equal(Wi, b[2 * i])
