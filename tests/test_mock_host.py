"""The library's host-side survey set-up against the FP64 oracle (no GPU needed):
the Schechter selection tables and mean numbers per magnitude bin (Sec. 5,
App. D) and the luminosity-dependent bias (Eq. rel_bias).  The library
integrates Phi by composite Gauss-Legendre quadrature and inverts the distance
by Newton's method; the oracle uses the closed-form incomplete gamma integral,
scipy's adaptive quadrature and a bracketing root finder."""
import os

import numpy as np
import pytest

from oracle import mock


@pytest.fixture(scope="module")
def lib():
    from paper_1306_1821_gb300 import bps
    from paper_1306_1821_gb300 import build as b
    if not os.path.exists(bps.LIB_PATH):
        b.build()
    return bps.load()


def test_schechter_tables_match_the_oracle(lib):
    from paper_1306_1821_gb300 import bps
    edges = np.array([-23.0, -21.8, -20.6, -19.4, -18.2, -17.0])
    r_max, n_r = 375.0, 97
    table, nb = bps.bps_schechter_tables(edges, r_max, n_r)
    ref = mock.selection_table(edges, r_max, n_r)
    assert np.max(np.abs(table - ref)) < 1e-10
    assert np.array_equal(table == 0.0, ref == 0.0) or np.max(np.abs(table - ref)) < 1e-12
    assert np.allclose(nb, mock.nbar_per_bin(edges, 1.0), rtol=1e-11, atol=0)
    # the paper's fifteen subsamples between M = -23 and -17
    e15 = np.linspace(-23.0, -17.0, 16)
    t15, nb15 = bps.bps_schechter_tables(e15, r_max, 9)
    assert np.allclose(nb15, mock.nbar_per_bin(e15, 1.0), rtol=1e-11, atol=0)
    assert np.all((t15 >= 0) & (t15 <= 1 + 1e-12))


def test_bias_law_matches_the_oracle(lib):
    from paper_1306_1821_gb300 import bps
    M = np.linspace(-23.0, -17.0, 15)
    assert np.allclose(bps.bps_bias_law(M), mock.bias_law(M), rtol=1e-15, atol=0)
    assert np.allclose(bps.bps_bias_law(M, b_star=2.0, M_star=-20.0, a=1.0, b=0.2, c=0.1),
                       mock.bias_law(M, 2.0, -20.0, 1.0, 0.2, 0.1), rtol=1e-15, atol=0)


def test_schechter_tables_reject_bad_arguments(lib):
    from paper_1306_1821_gb300 import bps
    with pytest.raises(bps.BpsError) as e:
        bps.bps_schechter_tables(np.array([-20.0, -21.0]), 100.0, 10)    # edges must increase
    assert e.value.status == bps.BPS_EINVAL
    with pytest.raises(bps.BpsError):
        bps.bps_schechter_tables(np.array([-21.0, -20.0]), 100.0, 1)
