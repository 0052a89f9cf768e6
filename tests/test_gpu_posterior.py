"""The posterior analysis of Secs. 6.2 and 7 (Figs. 6-11) accumulated on the
device (bps_posterior_moments / bps_posterior_read), through the C ABI, against
the plain definitions evaluated on the FP64 oracle chain's own samples: the
per-voxel ensemble mean and variance of delta, and the means and covariance of
(P, b, Nbar) from which the correlation matrices follow.

The GPU and oracle chains take the same draws; the comparison runs over
iterations whose Metropolis decisions all agree.  Tolerances: the fields agree
to ~1e-5 relative, so the mean map within 1e-4 relative L2, the variance map
within 1e-3; parameter means within 1e-4 relative, covariances within 1e-3 of
sqrt(var_i var_j)."""
import numpy as np
import pytest

from oracle import grid
from paper_1306_1821_gb300 import diagnostics
from tests.helpers import Problem, compare_chain, rel_l2

pytestmark = pytest.mark.gpu


def test_running_moments_match_the_oracle_chain():
    import torch

    from paper_1306_1821_gb300 import bps
    n_iter, nb, ns = 6, 8, 2
    pb = Problem(32, n_sub=ns, n_bins=nb, n_leapfrog=6, eps_max=0.15, jump_leapfrog=4, jump_eps_max=0.2)
    s = pb.gpu(seed=61, jump=1)
    try:
        with pytest.raises(bps.BpsError) as e:
            bps.bps_posterior_read(s.ctx, nb, ns)
        assert e.value.status == bps.BPS_ESTATE
        rec0 = bps.bps_gibbs_iterate(s.ctx, 2, s.rec_len)         # not accumulated
        bps.bps_posterior_moments(s.ctx, True)
        rec1 = bps.bps_gibbs_iterate(s.ctx, n_iter, s.rec_len)
        mean = torch.zeros((32,) * 3, dtype=torch.float64, device="cuda")
        var = torch.zeros_like(mean)
        pm, pc, n = bps.bps_posterior_read(s.ctx, nb, ns, mean, var)
        assert n == n_iter
        bps.bps_posterior_moments(s.ctx, False)
        bps.bps_gibbs_iterate(s.ctx, 1, s.rec_len)                # no longer accumulated
        assert bps.bps_posterior_read(s.ctx, nb, ns)[2] == n_iter
    finally:
        s.close()
    ch = pb.oracle_chain(seed=61, jump=True)
    done, _ = compare_chain(rec0, ch, 2)
    assert done == 2
    fields, params = [], []

    def keep(i, r):
        fields.append(grid.inverse(ch.delta_hat, 32))
        params.append(np.concatenate([r["P"], r["b"], r["nbar"]]))

    done, _ = compare_chain(rec1, ch, n_iter, on_iteration=keep)
    assert done == n_iter, "a decision fell inside the FP32 band; pick another seed"
    X = np.array(fields)
    assert rel_l2(mean.cpu().numpy(), X.mean(0)) < 1e-4
    assert rel_l2(var.cpu().numpy(), X.var(0)) < 1e-3
    Y = np.array(params)
    assert np.max(np.abs(pm / Y.mean(0) - 1)) < 1e-4
    cov = np.cov(Y.T, bias=True)
    sd = np.sqrt(np.outer(np.diag(cov), np.diag(cov)))
    assert np.max(np.abs(pc - cov) / np.where(sd > 0, sd, 1.0)) < 1e-3
    # the correlation blocks of Figs. 6 and 8
    blocks = diagnostics.parameter_blocks(diagnostics.correlation(pc), nb, ns)
    assert blocks["P-P"].shape == (nb, nb) and blocks["b-P"].shape == (ns, nb)
    assert np.allclose(np.diag(blocks["P-P"]), 1.0)
