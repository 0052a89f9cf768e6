"""Short chains of the named workloads against the FP64 oracle chain, through
the C ABI, with the jump on (Sec. 3.2 scan, Sec. 4.3 jump).

  * the 32^3 survey (L = 500 Mpc/h, one subsample with b = 1.2 held fixed and
    Nbar = 5, 40% sky with a linear radial fall-off, 16 bins, 10 leapfrog
    steps): five Gibbs iterations;
  * the 128^3 survey (L = 750 Mpc/h, six luminosity subsamples, 25% sky with
    exp(-(r/350)^2), 16 bins, 10 leapfrog steps): three iterations.

Per iteration the HMC Delta H agrees within 1e-3 and the Metropolis decisions
match (unless |Delta H + ln u| falls inside that band, after which the chains
are both valid but no longer comparable); P and Nbar agree within 1e-4
relative (the same Philox draws feed the same FP64 samplers; only the FP32
field sums differ), b within 1e-3.
"""
from dataclasses import replace

import pytest

from paper_1306_1821_gb300 import inputs
from tests.helpers import Problem, compare_chain

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,n_iter,min_compared", [("survey32", 5, 3), ("survey128", 3, 2)])
def test_workload_chain_matches_oracle(name, n_iter, min_compared):
    from paper_1306_1821_gb300 import bps
    wl = replace(inputs.WORKLOADS[name], jump=True)
    pb = Problem(wl.N, wl=wl)
    s = pb.gpu(seed=31, jump=1)
    try:
        rec = bps.bps_gibbs_iterate(s.ctx, n_iter, s.rec_len)
        ch = pb.oracle_chain(seed=31, jump=True)
        done, worst = compare_chain(rec, ch, n_iter)
        print(f"{name}: {done} iterations compared, max |dH - dH_oracle| = {worst:.2e}")
        assert done >= min_compared
    finally:
        s.close()
