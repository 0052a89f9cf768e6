"""Chain diagnostics (host-side analysis of recorded chains).

  * autocorrelation C(omega)_n of Sec. 6.1 (Eq. CORR_COEFF) and the paper's
    correlation length n_c, the first lag where C drops below 0.1;
  * effective sample size by Geyer's initial monotone sequence estimator
    (Geyer 1992, "Practical Markov chain Monte Carlo", Stat. Sci. 7): sums of
    adjacent autocorrelation pairs are truncated at the first non-positive pair
    and made monotone non-increasing.
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
