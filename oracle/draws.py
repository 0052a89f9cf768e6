"""Scalar random variates of the FP64 oracle (test infrastructure).

Each draw consumes Philox words at a fixed counter, so the CUDA library, which
implements the same published algorithms on its own, draws the same variates:

  * chi^2 of Sec. 4.2 (Eq. XI_SQUARE): x = 2 * Gamma(beta/2), with the Gamma
    variate by Marsaglia & Tsang, "A simple method for generating gamma
    variables", ACM TOMS 26 (2000): for shape a >= 1, d = a - 1/3,
    c = 1/sqrt(9 d); propose v = (1 + c z)^3 from a normal z and accept when
    ln u < z^2/2 + d - d v + d ln v; for a < 1 use Gamma(a+1) * U^(1/a).
    Attempt j of bin m reads block (m, iteration, STAGE_POWER, j): words 0,1 give
    z, word 2 gives u; word 3 of attempt 0 gives the a < 1 boost uniform.
    The paper's own recipe (sum of beta squared normals, Eq. post:posterior_of_x_1)
    has the same law; `chi2_sum_of_squares` keeps it as a cross-check.
  * the generalised inverse Gaussian of Sec. 3.6 (Eq. GIG_post), density
    proportional to x^(p-1) exp(-(A x + B / x) / 2).  The paper only cites a
    sampler; this one is the ratio-of-uniforms method with mode shift
    (Kinderman & Monahan 1977; for the GIG, Hoermann & Leydold 2014): with
    eta = sqrt(B/A), omega = sqrt(A B), y = x / eta (or its inverse when p < 0)
    has density h(y) ~ y^(lam-1) exp(-omega (y + 1/y) / 2), lam = |p|.  The
    acceptance region {0 < u <= sqrt(h(v/u + m)/h(m))} is enclosed in
    [0,1] x [v-, v+] with v+- the extremes of (y - m) sqrt(h(y)/h(m)), found by
    bisection on the derivative of its logarithm; everything is evaluated in
    log space relative to the mode m, which keeps |p| ~ 1e6 exact.
    Attempt j of subsample l reads block (l, iteration, STAGE_NBAR, j): word 0
    gives u, word 1 gives v.
"""
import math

import numpy as np

from . import philox

MAX_ATTEMPTS = 64


def _block(seed, iteration, stage, elem, sub):
    w = philox.words(seed, iteration, stage, sub, np.array([elem], dtype=np.uint64))
    return [x[0] for x in w]


def _u52(word):
    return (float(int(word) >> 12) + 0.5) * 2.0 ** -52


def _normal(wa, wb):
    return math.sqrt(-2.0 * math.log(_u52(wa))) * math.cos(2.0 * math.pi * _u52(wb))


def normal_draw(seed, iteration, stage, elem, sub=0):
    """One FP64 standard normal from words 0 and 1 of block (elem, iteration, stage, sub)."""
    w = _block(seed, iteration, stage, elem, sub)
    return _normal(w[0], w[1])


def gamma_mt(shape, seed, iteration, stage, elem):
    """Gamma(shape, 1) by Marsaglia-Tsang; returns (value, attempts used)."""
    a = float(shape)
    boost = a < 1.0
    aa = a + 1.0 if boost else a
    d = aa - 1.0 / 3.0
    c = 1.0 / math.sqrt(9.0 * d)
    val = d
    used = MAX_ATTEMPTS
    for j in range(MAX_ATTEMPTS):
        w = _block(seed, iteration, stage, elem, j)
        z = _normal(w[0], w[1])
        t = 1.0 + c * z
        if t <= 0.0:
            continue
        v = t * t * t
        u = _u52(w[2])
        if math.log(u) < 0.5 * z * z + d - d * v + d * math.log(v):
            val = d * v
            used = j + 1
            break
    if boost:
        w = _block(seed, iteration, stage, elem, 0)
        val *= math.exp(math.log(_u52(w[3])) / a)
    return val, used


def chi2_sum_of_squares(beta, rng):
    """Eq. post:posterior_of_x_1: x = sum of beta squared standard normals (integer beta)."""
    z = rng.standard_normal(int(beta))
    return float(np.sum(z * z))


def _gig_logh(y, lam, omega, m):
    """log h(y) - log h(m) for h(y) = y^(lam-1) exp(-omega (y + 1/y)/2)."""
    t = (y - m) / m
    return (lam - 1.0) * math.log1p(t) - 0.5 * omega * (y - m) * (1.0 - 1.0 / (y * m))


def _gig_dlogh(y, lam, omega):
    return (lam - 1.0) / y - 0.5 * omega + 0.5 * omega / (y * y)


def gig_mode(lam, omega):
    """Mode of h(y) = y^(lam-1) exp(-omega (y + 1/y)/2)."""
    q = lam - 1.0
    s = math.sqrt(q * q + omega * omega)
    return (q + s) / omega if q >= 0.0 else omega / (s - q)


def gig_bounds(lam, omega):
    """(m, v-, v+) of the mode-shifted ratio-of-uniforms rectangle."""
    m = gig_mode(lam, omega)

    def dphi(y):  # derivative of log|y - m| + log h(y) / 2
        return 1.0 / (y - m) + 0.5 * _gig_dlogh(y, lam, omega)

    # upper extreme: y in (m, inf); dphi goes from +inf to -omega/4
    step = m
    hi = m + step
    while dphi(hi) > 0.0:
        step *= 2.0
        hi = m + step
    lo = m
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if dphi(mid) > 0.0:
            lo = mid
        else:
            hi = mid
    yp = 0.5 * (lo + hi)
    vp = (yp - m) * math.exp(0.5 * _gig_logh(yp, lam, omega, m))
    # lower extreme: y in (0, m); dphi goes from a negative limit at 0+ ... to -inf at m-
    lo, hi = 0.0, m
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if dphi(mid) < 0.0:
            hi = mid
        else:
            lo = mid
    ym = 0.5 * (lo + hi)
    vm = (ym - m) * math.exp(0.5 * _gig_logh(ym, lam, omega, m)) if ym > 0.0 else -m
    return m, vm, vp


def gig_draw(p, A, B, seed, iteration, stage, elem):
    """GIG(p, A, B) variate by mode-shifted ratio of uniforms; returns (x, attempts)."""
    lam = abs(float(p))
    omega = math.sqrt(A * B)
    eta = math.sqrt(B / A)
    m, vm, vp = gig_bounds(lam, omega)
    y = m
    used = MAX_ATTEMPTS
    for j in range(MAX_ATTEMPTS):
        w = _block(seed, iteration, stage, elem, j)
        u = _u52(w[0])
        v = vm + (vp - vm) * _u52(w[1])
        yy = v / u + m
        if yy <= 0.0:
            continue
        if 2.0 * math.log(u) <= _gig_logh(yy, lam, omega, m):
            y = yy
            used = j + 1
            break
    x = eta * y if p >= 0.0 else eta / y
    return x, used
