"""Artificial surveys of Sec. 5, FP64 oracle (test infrastructure only).

Imported only by tests and the CPU baseline of the benchmark; shares no code
with the CUDA library, which generates the same surveys on the device.

  * True density field (Sec. 5, first paragraph): a zero-mean Gaussian field
    with covariance given by a power spectrum, delta = IFFT(A_k FFT(xi)) with
    xi white noise and A_k = sqrt(P(|k|) / V_cell) (App. C.1 convention, so
    E|delta_hat_k|^2 = N_vox P_k / V_cell as in the prior of Eq. dens_prior).
    A_k is given as a table over the integer |n|^2, A[0] = 0.  xi are the
    Philox voxel normals of stream (seed, 0, STAGE_MOCK_FIELD, 0).
  * Counts, Poisson form (the configs' data): N ~ Poisson(lambda) with
    lambda = (R Nbar) max(0, 1 + b delta), by inversion of the Poisson CDF in
    chunks of mean <= 32 (a sum of independent Poisson variates is Poisson
    with the summed mean).  Every decision is taken in FP64 with operations
    that IEEE 754 rounds exactly (+, -, *, /); e^-mu is evaluated by a fixed
    sequence of them (below), so that any implementation of this definition
    gives the same integers from the same inputs and Philox words.  Chunk j of
    voxel i of subsample l reads word j % 4 of block (i, j // 4,
    STAGE_MOCK_COUNTS, l).
  * Counts, Gaussian form (the paper's own noise, Sec. 5 and Eq.
    cov_mat_noise): N = Nbar R (1 + b delta) + eps, eps ~ N(0, Nbar R), from
    the FP64 normal of words 0, 1 of block (i, 0, STAGE_MOCK_COUNTS, l); the
    library stores integer counts, so the value is rounded to the nearest
    integer (halves up) and negative values are set to 0 (a stated reading).
  * Survey response (Sec. 5, Eq. for R^l_i): R = C(angle) f^l(r), here with a
    spherical-cap completeness about `axis` (the DR7 mask is not available)
    and the radial selection f^l sampled on a table of n_r radii in
    [0, r_max], linearly interpolated; R = 0 beyond r_max.
  * Radial selection from the Schechter function (Sec. 5 and App. D):
    f^l(r) = int_{M_lo(r)}^{M_hi(r)} Phi dM / int_{M_l}^{M_l+1} Phi dM with the
    absolute magnitudes a galaxy at distance r can have inside the apparent
    limits, M = m - mu(r), intersected with the subsample's bin.
    mu(r) = 5 log10(D_L / (Mpc/h)) + 25 (magnitudes M - 5 log10 h), D_L =
    (1 + z) r in a flat LCDM universe (Omega_m given) with r the comoving
    distance, no K-correction.
  * Mean numbers per bin: Nbar^l = Phi_* int_{M_l}^{M_l+1} Phi dM (Sec. 5).
  * Luminosity-dependent bias, Eq. rel_bias:
    b(M) = b_* (a + b 10^(0.4 (M_* - M)) + c (M - M_*)), at each bin's centre.
"""
import math

import numpy as np
from scipy import integrate, optimize, special

from . import grid, philox

STAGE_MOCK_FIELD = 8
STAGE_MOCK_COUNTS = 9
CHUNK_MEAN = 32.0        # largest mean of one inversion chunk
LAMBDA_MAX = 4096.0      # larger means are rejected (counts are 16-bit in the library)
MAX_STEPS = 200          # bound of one chunk's inversion search


# ------------------------------------------------------------------ field
def amplitude_table(N, box, spectrum):
    """A[n2] = sqrt(P(k) / V_cell), k = 2 pi sqrt(n2) / L, for n2 = 0..3 (N/2)^2 (A[0] = 0)."""
    n2 = np.arange(3 * (N // 2) ** 2 + 1, dtype=np.float64)
    k = 2.0 * np.pi * np.sqrt(n2) / box
    vc = (box / N) ** 3
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.sqrt(np.asarray(spectrum(k), dtype=np.float64) / vc)
    a[0] = 0.0
    return a


def field(N, amp, seed):
    """The true density field of one mock (FP64), from the Philox voxel normals."""
    xi = philox.voxel_normals(seed, 0, STAGE_MOCK_FIELD, 0, N ** 3).reshape(N, N, N)
    g = grid.Geometry(N, 1.0, 1)
    return grid.inverse(np.asarray(amp)[g.n2] * grid.forward(xi), N)


# ------------------------------------------------------------------ counts
def inv_factorials(n=10):
    """1/j! for j = 0..n, each the IEEE quotient of 1 by the exact integer j!."""
    return [1.0 / float(math.factorial(j)) for j in range(n + 1)]


def exp_neg(mu):
    """e^-mu for 0 <= mu <= 32 (arrays): mu scaled by 2^-10 (exact), the Taylor
    series of e^-x to degree 10 by Horner's rule (truncation below 1e-24 for
    x <= 1/32), then squared ten times.  Only IEEE-exact operations, in this
    order; relative accuracy ~1e-13."""
    x = np.asarray(mu, dtype=np.float64) * (2.0 ** -10)
    y = -x
    c = inv_factorials(10)
    s = np.full(x.shape, c[10])
    for j in range(9, -1, -1):
        s = s * y + c[j]
    for _ in range(10):
        s = s * s
    return s


def poisson_counts(lam, seed, sub, index=None):
    """Poisson variates of the flattened means `lam`; `index` gives each entry's
    voxel index (its Philox counter), by default its position."""
    lam = np.asarray(lam, dtype=np.float64).ravel()
    if np.any(lam > LAMBDA_MAX) or np.any(lam < 0):
        raise ValueError("means must lie in [0, 4096]")
    n = lam.size
    K = np.ceil(lam / CHUNK_MEAN)                    # chunks per voxel (0 where lam = 0)
    mu = np.where(K > 0, lam / np.maximum(K, 1.0), 0.0)
    e = exp_neg(mu)
    out = np.zeros(n, dtype=np.int64)
    vox = np.arange(n, dtype=np.uint64) if index is None else np.asarray(index, dtype=np.uint64).ravel()
    kmax = int(K.max()) if n else 0
    for j in range(kmax):
        act = K > j
        idx = np.nonzero(act)[0]
        w = philox.words(seed, j // 4, STAGE_MOCK_COUNTS, sub, vox[idx])[j % 4]
        u = philox.uniform52(w)
        m = mu[idx]
        p = e[idx].copy()
        F = p.copy()
        k = np.zeros(idx.size, dtype=np.int64)
        live = u > F
        for step in range(1, MAX_STEPS + 1):
            if not live.any():
                break
            li = np.nonzero(live)[0]
            k[li] = step
            p[li] = p[li] * m[li] / float(step)
            F[li] = F[li] + p[li]
            live[li] = u[li] > F[li]
        out[idx] += k
    return out


def mean_counts(delta, R, b, nbar, linear=False):
    """lambda = (R Nbar) max(0, 1 + b delta), FP64 from the given (FP32) arrays;
    linear=True keeps 1 + b delta unclipped (the paper's Gaussian data model)."""
    d = np.asarray(delta, dtype=np.float64)
    t = 1.0 + b * d
    if not linear:
        t = np.maximum(0.0, t)
    return (np.asarray(R, dtype=np.float64) * nbar) * t


def gaussian_counts(delta, R, b, nbar, seed, sub, index=None):
    """Counts under the paper's Gaussian noise model (rounded, clipped at 0);
    `index` as for poisson_counts."""
    m = mean_counts(delta, R, b, nbar, linear=True).ravel()
    var = np.asarray(R, dtype=np.float64).ravel() * nbar
    vox = np.arange(m.size, dtype=np.uint64) if index is None else np.asarray(index, dtype=np.uint64).ravel()
    w = philox.words(seed, 0, STAGE_MOCK_COUNTS, sub, vox)
    z = philox.normal64(w[0], w[1])
    x = m + np.sqrt(var) * z
    c = np.floor(x + 0.5)
    return np.where(var > 0, np.maximum(c, 0.0), 0.0).astype(np.int64)


def counts(delta, R, b, nbar, seed, noise="poisson"):
    """int64 [n_sub, N, N, N] counts of every subsample."""
    R = np.asarray(R)
    out = np.empty(R.shape, dtype=np.int64)
    for l in range(R.shape[0]):
        if noise == "poisson":
            out[l] = poisson_counts(mean_counts(delta, R[l], b[l], nbar[l]), seed, l).reshape(R.shape[1:])
        else:
            out[l] = gaussian_counts(delta, R[l], b[l], nbar[l], seed, l).reshape(R.shape[1:])
    return out


# ------------------------------------------------------------------ Schechter selection (App. D)
def schechter_phi(M, M_star=-20.44, alpha=-1.05):
    """Phi(M) of App. D with Phi_* = 1: 0.4 ln 10 x^(alpha+1) e^-x, x = 10^(0.4 (M_* - M))."""
    x = 10.0 ** (0.4 * (M_star - np.asarray(M, dtype=np.float64)))
    return 0.4 * math.log(10.0) * x ** (alpha + 1.0) * np.exp(-x)


def schechter_integral(M_lo, M_hi, M_star=-20.44, alpha=-1.05):
    """int_{M_lo}^{M_hi} Phi dM (Phi_* = 1) in closed form: with x = 10^(0.4 (M_* - M)),
    Phi dM = -x^alpha e^-x dx, so the integral is Gamma(alpha+1, x_hi) - Gamma(alpha+1, x_lo)
    (upper incomplete gamma).  For alpha + 1 = s < 0 the recurrence
    Gamma(s, x) = (Gamma(s+1, x) - x^s e^-x) / s gives it from s + 1 > 0."""
    M_lo = np.asarray(M_lo, dtype=np.float64)
    M_hi = np.asarray(M_hi, dtype=np.float64)
    s = alpha + 1.0

    def G(x):
        if s > 0:
            return special.gammaincc(s, x) * special.gamma(s)
        return (special.gammaincc(s + 1.0, x) * special.gamma(s + 1.0) - x ** s * np.exp(-x)) / s

    x_lo = 10.0 ** (0.4 * (M_star - M_lo))
    x_hi = 10.0 ** (0.4 * (M_star - M_hi))
    return np.where(M_hi > M_lo, G(x_hi) - G(x_lo), 0.0)


def comoving_distance(z, omega_m):
    """D_C(z) in Mpc/h, flat LCDM: (c/H0) int_0^z dz' / sqrt(Om (1+z')^3 + 1 - Om)."""
    c_h0 = 299792.458 / 100.0
    f = lambda t: 1.0 / math.sqrt(omega_m * (1.0 + t) ** 3 + 1.0 - omega_m)
    return c_h0 * integrate.quad(f, 0.0, z, epsabs=0, epsrel=1e-13)[0]


def redshift_of(r, omega_m):
    if r <= 0.0:
        return 0.0
    return optimize.brentq(lambda z: comoving_distance(z, omega_m) - r, 0.0, 10.0, xtol=1e-15, rtol=1e-15)


def distance_modulus(r, omega_m):
    """mu = 5 log10(D_L / (Mpc/h)) + 25, D_L = (1 + z) r (magnitudes M - 5 log10 h)."""
    z = redshift_of(r, omega_m)
    return 5.0 * math.log10((1.0 + z) * r) + 25.0


def selection(r, M_l, M_u, m_bright=14.5, m_faint=17.77, M_star=-20.44, alpha=-1.05, omega_m=0.24):
    """f^l(r) of Sec. 5 for the magnitude bin [M_l, M_u] (brightest first)."""
    if r <= 0.0:
        return 0.0
    mu = distance_modulus(r, omega_m)
    lo = max(M_l, m_bright - mu)
    hi = min(M_u, m_faint - mu)
    if not hi > lo:
        return 0.0
    return float(schechter_integral(lo, hi, M_star, alpha) / schechter_integral(M_l, M_u, M_star, alpha))


def selection_table(M_edges, r_max, n_r, **kw):
    """[n_sub][n_r] samples of f^l at r_j = j r_max / (n_r - 1)."""
    r = np.arange(n_r) * (r_max / (n_r - 1))
    return np.array([[selection(x, M_edges[l], M_edges[l + 1], **kw) for x in r]
                     for l in range(len(M_edges) - 1)])


def nbar_per_bin(M_edges, phi_star, M_star=-20.44, alpha=-1.05):
    """Nbar^l = Phi_* int over the l-th magnitude bin of Phi (Sec. 5)."""
    e = np.asarray(M_edges, dtype=np.float64)
    return phi_star * schechter_integral(e[:-1], e[1:], M_star, alpha)


def bias_law(M, b_star=1.2, M_star=-20.83, a=0.895, b=0.105, c=-0.040):
    """Eq. rel_bias: b(M) = b_* (a + b 10^(0.4 (M_* - M)) + c (M - M_*))."""
    M = np.asarray(M, dtype=np.float64)
    return b_star * (a + b * 10.0 ** (0.4 * (M_star - M)) + c * (M - M_star))


# ------------------------------------------------------------------ response
def response(N, box, f_sky, axis, table, r_max):
    """R [n_sub, N, N, N] float32: spherical cap (cos theta >= 1 - 2 f_sky about
    `axis`) inside r <= r_max, times the linearly interpolated selection table."""
    dx = box / N
    cc = (np.arange(N) + 0.5) * dx - box / 2.0
    x, y, z = np.meshgrid(cc, cc, cc, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    ax = np.asarray(axis, dtype=np.float64)
    ax = ax / math.sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2])
    proj = ax[0] * x + ax[1] * y + ax[2] * z
    cos_t = np.where(r > 0, proj / np.where(r > 0, r, 1.0), 1.0)
    inside = (cos_t >= 1.0 - 2.0 * f_sky) & (r <= r_max)
    table = np.asarray(table, dtype=np.float64)
    n_r = table.shape[1]
    t = np.minimum(r / r_max * (n_r - 1), n_r - 1)
    j = np.minimum(np.floor(t).astype(np.int64), n_r - 2)
    w = t - j
    out = np.empty((table.shape[0], N, N, N), dtype=np.float32)
    for l in range(table.shape[0]):
        f = table[l][j] * (1.0 - w) + table[l][j + 1] * w
        out[l] = np.where(inside, f, 0.0).astype(np.float32)
    return out
