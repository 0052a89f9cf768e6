"""Counter-based random streams of the FP64 oracle (test infrastructure only).

Philox4x64-10 of Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy
as 1, 2, 3" (SC'11), written from its published definition: a 4-word counter and
a 2-word key, ten rounds of two 64x64->128 multiplies, key bumped by the two
Weyl constants between rounds.  The CUDA library implements the same generator
on its own; the two share no code.  Every random number the sampler draws is a
pure function of (seed, counter), so the oracle can replay any draw the GPU
makes.

Counter layout used by the sampler (all words 64-bit):
    ctr = (element_block, gibbs_iteration, stage, sub_index), key = (seed, 0)

Stages (one per random decision of the multiple-block scan, Sec. 3.2):
    STAGE_MOMENTUM   HMC momentum field xi (Sec. 4.1.1: momenta redrawn each move)
    STAGE_HMC        HMC step-size fraction and accept uniform (Sec. 4.1.2, Eq. acceptance_rule)
    STAGE_POWER      chi^2 draws of the power spectrum (Sec. 4.2)
    STAGE_BIAS       normal bias draws (Sec. 3.5, App. B)
    STAGE_NBAR       GIG draws of the normalisations (Sec. 3.6, App. A)
    STAGE_JUMP_MOM   momenta of the deterministic-jump HMC (Sec. 4.3, App. C)
    STAGE_JUMP       step-size fraction and accept uniform of the jump HMC

This module is imported only by tests, the smoke check and the CPU baseline leg
of the benchmark.
"""
import numpy as np

M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15
W1 = 0xBB67AE8584CAA73B
_MASK32 = np.uint64(0xFFFFFFFF)

STAGE_MOMENTUM = 1
STAGE_HMC = 2
STAGE_POWER = 3
STAGE_BIAS = 4
STAGE_NBAR = 5
STAGE_JUMP_MOM = 6
STAGE_JUMP = 7


def _mulhilo64(a, b):
    """Full 128-bit product of uint64 arrays a and scalar b, as (hi, lo)."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.uint64(b)
    a_lo, a_hi = a & _MASK32, a >> np.uint64(32)
    b_lo, b_hi = b & _MASK32, b >> np.uint64(32)
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> np.uint64(32)) + (lh & _MASK32) + (hl & _MASK32)
    hi = hh + (lh >> np.uint64(32)) + (hl >> np.uint64(32)) + (mid >> np.uint64(32))
    lo = a * b  # wraps modulo 2^64
    return hi, lo


def philox4x64(c0, c1, c2, c3, k0, k1):
    """Philox4x64-10 bijection.  Counter words may be arrays (broadcast)."""
    with np.errstate(over="ignore"):
        x0, x1, x2, x3 = np.broadcast_arrays(*(np.asarray(c, dtype=np.uint64) for c in (c0, c1, c2, c3)))
        x0, x1, x2, x3 = (x.copy() for x in (x0, x1, x2, x3))
        ka = int(k0) & 0xFFFFFFFFFFFFFFFF
        kb = int(k1) & 0xFFFFFFFFFFFFFFFF
        for _ in range(10):
            hi0, lo0 = _mulhilo64(x0, M0)
            hi1, lo1 = _mulhilo64(x2, M1)
            x0, x1, x2, x3 = hi1 ^ x1 ^ np.uint64(ka), lo1, hi0 ^ x3 ^ np.uint64(kb), lo0
            ka = (ka + W0) & 0xFFFFFFFFFFFFFFFF
            kb = (kb + W1) & 0xFFFFFFFFFFFFFFFF
    return x0, x1, x2, x3


def words(seed, iteration, stage, sub, blocks):
    """The four output words for element blocks `blocks` (array) of one stream."""
    return philox4x64(blocks, iteration, stage, sub, seed, 0)


def uniform52(w):
    """FP64 uniform in (0,1) from a 64-bit word: ((w >> 12) + 1/2) * 2^-52.

    Every step is exact in double precision (the sum needs at most 53
    significant bits), so the value is identical on any IEEE machine; the range
    is [2^-53, 1 - 2^-53].
    """
    w = np.asarray(w, dtype=np.uint64)
    return ((w >> np.uint64(12)).astype(np.float64) + 0.5) * 2.0 ** -52


def normal64(w_a, w_b):
    """FP64 standard normal from two words: Box-Muller cosine branch (Box & Muller 1958)."""
    u1 = uniform52(w_a)
    u2 = uniform52(w_b)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def uniform24_pair(w):
    """The two FP32-representable uniforms the momentum transform uses.

    From the low and high 32-bit halves h of a word: fl32(fl32(h) * 2^-32 + 2^-33),
    evaluated in IEEE single precision with round-to-nearest, so the value is
    identical on any IEEE machine.  Range [2^-33, 1].
    """
    w = np.asarray(w, dtype=np.uint64)
    lo = (w & _MASK32).astype(np.uint32).astype(np.float32)
    hi = (w >> np.uint64(32)).astype(np.uint32).astype(np.float32)
    s = np.float32(2.0 ** -32)
    o = np.float32(2.0 ** -33)
    return lo * s + o, hi * s + o


def voxel_normals(seed, iteration, stage, sub, n):
    """n standard normals for a real field, element i from block i//8.

    Word j = (i % 8) // 2 of block i // 8 gives a Box-Muller pair from its two
    FP32 uniforms (u1 from the low half, u2 from the high half): element i takes
    the cosine branch when i is even and the sine branch when i is odd.  The
    oracle evaluates the transform in FP64 from the same uniforms.
    """
    nb = (n + 7) // 8
    blocks = np.arange(nb, dtype=np.uint64)
    ws = words(seed, iteration, stage, sub, blocks)
    out = np.empty(nb * 8, dtype=np.float64)
    for j in range(4):
        u1, u2 = uniform24_pair(ws[j])
        r = np.sqrt(-2.0 * np.log(u1.astype(np.float64)))
        t = 2.0 * np.pi * u2.astype(np.float64)
        out[2 * j::8] = r * np.cos(t)
        out[2 * j + 1::8] = r * np.sin(t)
    return out[:n]
