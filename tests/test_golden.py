"""The paper's printed numbers for its artificial survey (Sec. 5, Sec. 6.2),
held as cited text fixtures under tests/golden/, against the oracle, the
stored workload tables and the library's host-side survey set-up.

  * `sec5_setup.txt`: constants the paper prints, one citation per line.
  * `schechter15.txt`: the fifteen-bin tables (edges, Nbar^l, b^l, Phi_*),
    written by tests/golden/schechter15.py from those constants and the oracle.

A mistyped constant in the oracle, the workload or the library's defaults, or a
stored table that drifted from its definition, fails here.
"""
import inspect
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import mock
from paper_1306_1821_gb300 import bps, inputs
from tests.golden import schechter15 as g15

SETUP = g15.read_setup()
V = {k: v[0] for k, v in SETUP.items()}
PHI_STAR, ROWS = g15.read_table()


def defaults(fn):
    return {k: p.default for k, p in inspect.signature(fn).parameters.items()
            if p.default is not inspect.Parameter.empty}


def test_fixture_is_cited_and_consistent():
    for name, (_, cite) in SETUP.items():
        assert cite.startswith("Sec. "), name
    assert V["n_vox"] == V["n_side"] ** 3                       # Sec. 5: 128^3 = 2097152
    assert V["M_max"] < V["M_min"]                              # brightest magnitude is the most negative
    assert V["m_bright"] < V["m_faint"]
    # Eq. rel_bias: with the printed fit a + b = 1, so b(M_*) = b_* exactly
    assert V["bias_a"] + V["bias_b"] == pytest.approx(1.0, abs=1e-15)


def test_oracle_defaults_are_the_papers_constants():
    sch = dict(M_star=V["schechter_M_star"], alpha=V["schechter_alpha"])
    for fn in (mock.schechter_phi, mock.schechter_integral, mock.nbar_per_bin):
        assert {k: defaults(fn)[k] for k in sch} == sch, fn.__name__
    assert defaults(mock.selection) == dict(sch, m_bright=V["m_bright"], m_faint=V["m_faint"],
                                            omega_m=defaults(mock.selection)["omega_m"])
    assert defaults(mock.bias_law) == dict(b_star=V["bias_b_star"], M_star=V["bias_M_star"],
                                           a=V["bias_a"], b=V["bias_b"], c=V["bias_c"])
    assert float(mock.bias_law(V["bias_M_star"])) == pytest.approx(V["bias_b_star"], rel=1e-15)


def test_library_defaults_are_the_papers_constants():
    bias = dict(b_star=V["bias_b_star"], M_star=V["bias_M_star"], a=V["bias_a"], b=V["bias_b"], c=V["bias_c"])
    assert bps.BIAS_LAW_PAPER == bias
    assert defaults(bps.bps_bias_law) == bias
    sch = dict(M_star=V["schechter_M_star"], alpha=V["schechter_alpha"], m_bright=V["m_bright"],
               m_faint=V["m_faint"])
    assert {k: bps.SCHECHTER_SDSS[k] for k in sch} == sch
    assert {k: defaults(bps.bps_schechter_tables)[k] for k in sch} == sch
    assert bps.SCHECHTER_SDSS["omega_m"] == defaults(bps.bps_schechter_tables)["omega_m"]


def test_schechter_workload_is_the_papers_setup():
    wl = inputs.WORKLOADS["schechter128"]
    assert wl.N == V["n_side"] and wl.N ** 3 == V["n_vox"]
    assert wl.box == V["box"]
    assert wl.n_sub == V["n_sub"]
    e = np.asarray(wl.extra["M_edges"])
    assert e[0] == V["M_max"] and e[-1] == pytest.approx(V["M_min"], abs=1e-12)
    assert np.allclose(np.diff(e), (V["M_min"] - V["M_max"]) / V["n_sub"], rtol=0, atol=1e-12)
    # Sec. 6.2: the bias held at unity is that of the bin centred on M = -20.4
    l = wl.fixed_bias
    assert 0.5 * (e[l] + e[l + 1]) == pytest.approx(V["fixed_bias_M"], abs=1e-12)


def test_stored_tables_are_the_golden_tables():
    assert len(ROWS) == V["n_sub"]
    assert inputs.SCHECHTER15_PHI_STAR == PHI_STAR
    assert inputs.SCHECHTER15_EDGES == [r[1] for r in ROWS] + [ROWS[-1][2]]
    assert inputs.SCHECHTER15_NBAR == [r[3] for r in ROWS]
    assert inputs.SCHECHTER15_B == [r[4] for r in ROWS]


def test_golden_tables_follow_from_the_oracle():
    phi, rows = g15.compute(SETUP)
    assert phi == pytest.approx(PHI_STAR, rel=1e-13)
    got = np.array([r[1:] for r in rows])
    ref = np.array([r[1:] for r in ROWS])
    assert np.allclose(got, ref, rtol=1e-13, atol=0)


def test_golden_tables_against_quadrature_of_phi():
    # Nbar^l by adaptive quadrature of Phi itself (App. D), not the incomplete-gamma closed form
    phi_sch = lambda M: 0.4 * math.log(10.0) * PHI_STAR * (
        10.0 ** (0.4 * (V["schechter_M_star"] - M))) ** (V["schechter_alpha"] + 1.0) * math.exp(
        -(10.0 ** (0.4 * (V["schechter_M_star"] - M))))
    for l, lo, hi, nb, b in ROWS:
        q = integrate.quad(phi_sch, lo, hi, epsabs=0, epsrel=1e-13)[0]
        assert nb == pytest.approx(q, rel=1e-11), l
        Mc = 0.5 * (lo + hi)
        x = 10.0 ** (0.4 * (V["bias_M_star"] - Mc))
        assert b == pytest.approx(V["bias_b_star"] * (V["bias_a"] + V["bias_b"] * x + V["bias_c"] * (Mc - V["bias_M_star"])),
                                  rel=1e-14), l
    assert ROWS[-1][3] == g15.NBAR_FAINTEST
    nb = np.array([r[3] for r in ROWS])
    b = np.array([r[4] for r in ROWS])
    assert np.all(np.diff(b) < 0)          # brighter subsamples are more biased
    assert np.all(np.diff(nb) > 0)         # and rarer, over this magnitude range


@pytest.fixture(scope="module")
def lib():
    from paper_1306_1821_gb300 import build as b
    if not os.path.exists(bps.LIB_PATH):
        b.build()
    return bps.load()


def test_library_host_setup_gives_the_golden_tables(lib):
    e = np.array([r[1] for r in ROWS] + [ROWS[-1][2]])
    _, nb_rel = bps.bps_schechter_tables(e, 375.0, 9)
    assert np.allclose(PHI_STAR * nb_rel, [r[3] for r in ROWS], rtol=1e-11, atol=0)
    b = bps.bps_bias_law(0.5 * (e[:-1] + e[1:]))
    assert np.allclose(b, [r[4] for r in ROWS], rtol=1e-14, atol=0)
