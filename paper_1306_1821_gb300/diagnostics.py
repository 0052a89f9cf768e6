"""Chain diagnostics (host-side analysis of recorded chains).

  * autocorrelation C(omega)_n of Sec. 6.1 (Eq. CORR_COEFF) and the paper's
    correlation length n_c, the first lag where C drops below 0.1;
  * effective sample size by Geyer's initial monotone sequence estimator
    (Geyer 1992, "Practical Markov chain Monte Carlo", Stat. Sci. 7): sums of
    adjacent autocorrelation pairs are truncated at the first non-positive pair
    and made monotone non-increasing;
  * the posterior analysis of Secs. 6.2 and 7 (Figs. 6-11) from the moments the
    library accumulates on the device (bps_posterior_moments / _read): the
    correlation matrices of P-P, b-P, Nbar-P and b-Nbar, and two-dimensional
    marginal histograms of any pair of recorded chain quantities.
"""
import numpy as np


def autocorr(x, max_lag=None):
    """C_n for n = 0..max_lag (Eq. CORR_COEFF, normalised by the sample variance)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    max_lag = n - 1 if max_lag is None else min(max_lag, n - 1)
    y = x - x.mean()
    v = np.dot(y, y) / n
    if v <= 0:
        return np.ones(max_lag + 1)
    f = np.fft.rfft(y, 2 * n)
    ac = np.fft.irfft(f * np.conj(f))[: max_lag + 1] / n
    return ac / v


def correlation_length(x, threshold=0.1):
    """First lag at which the autocorrelation falls below `threshold` (Sec. 6.1)."""
    c = autocorr(x)
    idx = np.nonzero(c < threshold)[0]
    return int(idx[0]) if idx.size else len(c)


def ess_geyer(x):
    """Effective sample size by the initial monotone sequence estimator."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    if n < 4:
        return float(n)
    c = autocorr(x)
    pairs = []
    for k in range(0, (n - 1) // 2):
        g = c[2 * k] + c[2 * k + 1]
        if g <= 0:
            break
        pairs.append(g)
    if not pairs:
        return float(n)
    g = np.minimum.accumulate(np.array(pairs))
    tau = -1.0 + 2.0 * g.sum()
    return float(n / max(tau, 1e-12))


def correlation(cov):
    """Correlation matrix cov_ij / sqrt(cov_ii cov_jj) (zero where a variance is zero)."""
    cov = np.asarray(cov, dtype=np.float64)
    sd = np.sqrt(np.maximum(np.diag(cov), 0.0))
    den = np.outer(sd, sd)
    return np.where(den > 0, cov / np.where(den > 0, den, 1.0), 0.0)


def parameter_blocks(corr, n_bins, n_sub):
    """The blocks of the parameter correlation matrix (order P, b, Nbar) shown in
    Figs. 6 and 8: P-P, b-P, Nbar-P and b-Nbar."""
    P = slice(0, n_bins)
    b = slice(n_bins, n_bins + n_sub)
    nb = slice(n_bins + n_sub, n_bins + 2 * n_sub)
    return {"P-P": corr[P, P], "b-P": corr[b, P], "Nbar-P": corr[nb, P], "b-Nbar": corr[b, nb]}


def marginal_2d(x, y, bins=30, ranges=None):
    """Normalised two-dimensional histogram of paired samples (Fig. 7's marginal
    posteriors of pairs of modes); returns (density, x edges, y edges)."""
    h, ex, ey = np.histogram2d(np.asarray(x), np.asarray(y), bins=bins, range=ranges, density=True)
    return h, ex, ey
