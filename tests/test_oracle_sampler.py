"""Pin of the oracle's whole multiple-block sampler (Sec. 3.2, Eq. multiblock,
Fig. 1): the scan HMC(delta) -> P -> [P-delta jump] -> b -> Nbar -> rebuild,
with its state threading, against an exact posterior that does not use any
part of the sampler.

On a 4^3 grid with one galaxy subsample and the bias held fixed, the density
field can be integrated out in closed form.  Under the data model of Eq.
data_model with the Gaussian noise of Eq. cov_mat_noise (variance Nbar R per
voxel, Eq. LH_all_dataset) and the Gaussian prior of Eq. dens_prior, the
observed counts are jointly Gaussian given (P, Nbar):

    d ~ N(Nbar R,  diag(Nbar R) + Nbar^2 b^2 diag(R) S(P) diag(R)),

over the voxels with R > 0, with S(P) the prior covariance of Eq. dens_prior
(Fourier eigenvalues P_m / V_cell, zero on the k = 0 mode).  With the priors of
the sampler (P^-alpha per bin, Sec. 3.4, here alpha = 0; flat in Nbar > 0,
Sec. 3.6) this gives
the joint posterior of (P, Nbar) up to a constant; a quadrature grid over it
gives the marginal moments.  Oracle Gibbs chains, once with the jump of
Sec. 4.3 and once without, must reproduce them within 3.5 Monte Carlo standard
errors (batch means), for one power bin (2D quadrature) and two bins (3D).
"""
import math
import multiprocessing
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

from oracle import gibbs, grid

N = 4
BOX = 20.0          # V_cell = 125
B_FIXED = 1.2
NBAR_TRUE = 10.0
P_TRUE = 60.0       # voxel variance ~ 0.47
# Flat prior on P (alpha = 0, Sec. 3.4).  Under the Jeffreys prior (alpha = 1)
# the marginal posterior of ln P tends to a constant as P -> 0 (the likelihood
# no longer depends on P there), so it is improper and has no moments to pin.
ALPHA = 0.0
BURN = 300
N_ITER = 4000
N_BATCH = 30


def make_data(seed, n_bins):
    """Counts drawn from the paper's Gaussian data model; R in [0.4, 1] with
    about one voxel in eight masked (R = 0, count 0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = grid.Geometry(N, BOX, n_bins)
    il = np.where(g.bin >= 0, 1.0, 0.0) * (P_TRUE / g.Vc)
    xi = rng.standard_normal((N, N, N))
    delta = grid.inverse(np.sqrt(il) * grid.forward(xi), N)
    R = rng.uniform(0.4, 1.0, (N, N, N))
    R[rng.random((N, N, N)) < 0.12] = 0.0
    lam = NBAR_TRUE * R * (1.0 + B_FIXED * delta)
    d = lam + np.sqrt(NBAR_TRUE * R) * rng.standard_normal((N, N, N))
    d = np.where(R > 0, d, 0.0)
    return g, d[None], R[None]


def unit_covariances(g):
    """S_m for unit power in bin m: (S_m)_ij = (1 / (N_vox V_cell)) sum_{k in m} cos(k (x_i - x_j)),
    summed over the full grid (the prior covariance of Eq. dens_prior is sum_m P_m S_m)."""
    i = np.arange(N)
    s = np.where(i <= N // 2, i, i - N)
    nx, ny, nz = np.meshgrid(s, s, s, indexing="ij")
    kv = np.stack([nx.ravel(), ny.ravel(), nz.ravel()], -1)
    b = grid.bin_of_n2((kv ** 2).sum(1), N, g.n_bins)
    x = np.stack(np.meshgrid(i, i, i, indexing="ij"), -1).reshape(-1, 3)
    ph = 2.0 * np.pi * (x @ kv.T) / N                       # [voxel, mode]
    out = []
    for m in range(g.n_bins):
        sel = b == m
        c, sn = np.cos(ph[:, sel]), np.sin(ph[:, sel])
        out.append((c @ c.T + sn @ sn.T) / (g.Nv * g.Vc))
    return out


def log_posterior(g, d, R, Ps, nbars, alpha=ALPHA):
    """log p(P, Nbar | d) + const on the grid Ps [n_P, n_bins] x nbars [n_nbar]."""
    obs = R[0].ravel() > 0
    r = R[0].ravel()[obs]
    y = d[0].ravel()[obs]
    Sm = [S[np.ix_(obs, obs)] for S in unit_covariances(g)]
    nbars = np.asarray(nbars, dtype=np.float64)
    out = np.empty((len(Ps), len(nbars)))
    for i, P in enumerate(Ps):
        S = sum(p * s for p, s in zip(P, Sm))
        RSR = (r[:, None] * S * r[None, :]) * B_FIXED ** 2
        C = nbars[:, None, None] * np.diag(r)[None] + (nbars ** 2)[:, None, None] * RSR[None]
        L = np.linalg.cholesky(C)                                     # one per Nbar
        z = np.linalg.solve(L, (y[None, :] - nbars[:, None] * r[None, :])[..., None])[..., 0]
        logdet = np.sum(np.log(np.diagonal(L, axis1=1, axis2=2)), 1)
        out[i] = -0.5 * np.sum(z * z, 1) - logdet - alpha * np.sum(np.log(P))
    return out


def posterior_moments(g, d, R, p_axes, nbars):
    """Posterior means of P_m, ln P_m and Nbar by quadrature on a tensor grid in
    (ln P_0, ..., ln P_{n-1}, Nbar); the measure dP = P d ln P is included."""
    mesh = np.meshgrid(*p_axes, indexing="ij")
    Ps = np.stack([np.exp(m.ravel()) for m in mesh], -1)
    lp = log_posterior(g, d, R, Ps, nbars) + np.sum(np.log(Ps), 1)[:, None]
    w = np.exp(lp - lp.max())
    w /= w.sum()
    res = {}
    for m in range(g.n_bins):
        res[f"P{m}"] = float(np.sum(w * Ps[:, m:m + 1]))
        res[f"lnP{m}"] = float(np.sum(w * np.log(Ps[:, m:m + 1])))
        res[f"sdlnP{m}"] = math.sqrt(float(np.sum(w * np.log(Ps[:, m:m + 1]) ** 2)) - res[f"lnP{m}"] ** 2)
    res["nbar"] = float(np.sum(w * nbars[None, :]))
    res["sdnbar"] = math.sqrt(float(np.sum(w * nbars[None, :] ** 2)) - res["nbar"] ** 2)
    # the posterior mass must lie inside the grid; with alpha = 0 the density
    # in ln P_m falls off only as P_m towards P_m -> 0 in a bin with few modes,
    # so the grid reaches far down and the mass left beyond it is below 1e-5
    edge = w.reshape(*[len(a) for a in p_axes], len(nbars))
    for ax in range(edge.ndim):
        e = np.moveaxis(edge, ax, 0)
        assert e[0].sum() < 1e-6 and e[-1].sum() < 1e-6, "quadrature grid too narrow"
    return res


def run_chain(args):
    """One oracle chain (runs in a spawned worker); returns its P and Nbar records."""
    seed_data, n_bins, jump, seed = args
    g, d, R = make_data(seed_data, n_bins)
    P0 = np.full(n_bins, P_TRUE)
    ch = gibbs.Chain(g, d, R, P0, [B_FIXED], [NBAR_TRUE], alpha=ALPHA, n_leapfrog=8, eps_max=0.5, jump=jump,
                     jump_leapfrog=6, jump_eps_max=0.5, fixed_bias=0, seed=seed)
    P = np.empty((N_ITER, n_bins))
    nb = np.empty(N_ITER)
    acc = 0
    for it in range(N_ITER):
        rec = ch.iterate()
        P[it] = rec["P"]
        nb[it] = rec["nbar"][0]
        acc += rec["hmc"]["accepted"]
    return P, nb, acc / N_ITER


def batch_se(x):
    x = np.asarray(x)[BURN:]
    n = len(x) // N_BATCH * N_BATCH
    bm = x[:n].reshape(N_BATCH, -1).mean(1)
    return float(x.mean()), float(bm.std(ddof=1) / math.sqrt(N_BATCH))


CASES = [(21, 1, True, 7), (21, 1, False, 8), (22, 2, True, 9), (22, 2, False, 10)]


@pytest.fixture(scope="module")
def chains():
    ctx = multiprocessing.get_context("spawn")
    with ProcessPoolExecutor(max_workers=len(CASES), mp_context=ctx) as ex:
        out = list(ex.map(run_chain, CASES))
    return dict(zip(CASES, out))


def quadrature(seed_data, n_bins):
    g, d, R = make_data(seed_data, n_bins)
    if n_bins == 1:
        axes = [np.linspace(math.log(P_TRUE) - 2.5, math.log(P_TRUE) + 2.5, 201)]
        nbars = np.linspace(4.0, 14.0, 201)
    else:
        axes = [np.linspace(math.log(P_TRUE) - 8.0, math.log(P_TRUE) + 4.0, 97),
                np.linspace(math.log(P_TRUE) - 2.5, math.log(P_TRUE) + 4.5, 57)]
        nbars = np.linspace(3.0, 16.0, 53)
    return posterior_moments(g, d, R, axes, nbars)


@pytest.mark.slow
@pytest.mark.parametrize("seed_data,n_bins", [(21, 1), (22, 2)])
def test_gibbs_chains_match_the_marginal_posterior(chains, seed_data, n_bins):
    ref = quadrature(seed_data, n_bins)
    for jump in (True, False):
        key = next(k for k in CASES if k[0] == seed_data and k[1] == n_bins and k[2] == jump)
        P, nb, acc = chains[key]
        assert acc > 0.7
        for m in range(n_bins):
            mu, se = batch_se(np.log(P[:, m]))
            assert abs(mu - ref[f"lnP{m}"]) < 3.5 * se, (jump, m, mu, ref[f"lnP{m}"], se)
            # the spread of the marginal as well (a scan that mixed up its
            # conditionals would get the width wrong before the mean)
            sd = float(np.log(P[BURN:, m]).std())
            assert abs(sd / ref[f"sdlnP{m}"] - 1.0) < 0.12, (jump, m, sd, ref[f"sdlnP{m}"])
        mu, se = batch_se(nb)
        assert abs(mu - ref["nbar"]) < 3.5 * se, (jump, mu, ref["nbar"], se)
        sd = float(nb[BURN:].std())
        assert abs(sd / ref["sdnbar"] - 1.0) < 0.12, (jump, sd, ref["sdnbar"])


def test_marginal_likelihood_matches_brute_force_integral_over_delta():
    """The closed-form marginal used above, checked against the product of the
    likelihood and the prior integrated over delta by Monte Carlo importance
    sampling on a 2^3 grid: a check of the formula, not of the sampler."""
    n = 2
    g = grid.Geometry(n, 10.0, 1)
    rng = np.random.Generator(np.random.PCG64(4))
    R = rng.uniform(0.5, 1.0, (n, n, n))
    d = 5.0 * R + rng.standard_normal((n, n, n))
    P, nb = 40.0, 4.0
    # prior covariance of delta on the grid: (P / V_cell) (I - 11^T / N_vox)
    Sv = (P / g.Vc) * (np.eye(8) - 1.0 / 8.0)
    r = R.ravel()
    C = nb * np.diag(r) + nb * nb * B_FIXED ** 2 * (r[:, None] * Sv * r[None, :])
    sign, logdet = np.linalg.slogdet(2 * np.pi * C)
    y = d.ravel() - nb * r
    closed = -0.5 * y @ np.linalg.solve(C, y) - 0.5 * logdet
    # Monte Carlo: E_delta~prior [ prod_i N(d_i; nb r_i (1 + b delta_i), nb r_i) ]
    w, V = np.linalg.eigh(Sv)
    z = rng.standard_normal((400000, 8))
    delta = (z * np.sqrt(np.maximum(w, 0.0))) @ V.T
    mu = nb * r * (1.0 + B_FIXED * delta)
    ll = -0.5 * np.sum((d.ravel() - mu) ** 2 / (nb * r), 1) - 0.5 * np.sum(np.log(2 * np.pi * nb * r))
    mx = ll.max()
    mc = mx + math.log(np.mean(np.exp(ll - mx)))
    assert abs(mc - closed) < 0.02
