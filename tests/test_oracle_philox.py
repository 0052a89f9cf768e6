"""Pins of the oracle's Philox generator and uniform / normal transforms."""
import numpy as np
import pytest
from scipy import stats

from oracle import philox


@pytest.mark.parametrize("key,counter", [(0, 0), (12345, 7), (2**64 - 1, 2**63 + 5), (0xDEADBEEF, 2**64 - 2)])
def test_philox_matches_numpy_bitgenerator(key, counter):
    # numpy's Philox is an independent implementation of Philox4x64-10; its
    # stream with counter c yields philox(c + 1), philox(c + 2), ... (256-bit
    # counter, little-endian words, carry between words).
    bg = np.random.Philox(key=key, counter=counter)
    ref = bg.random_raw(4 * 6).reshape(6, 4)
    for j in range(6):
        c = counter + 1 + j
        w = [c & (2**64 - 1), (c >> 64) & (2**64 - 1), 0, 0]
        out = philox.philox4x64(w[0], w[1], w[2], w[3], key & (2**64 - 1), (key >> 64) & (2**64 - 1))
        assert [int(x) for x in out] == [int(x) for x in ref[j]]


def test_philox_vectorised_equals_scalar():
    blocks = np.arange(37, dtype=np.uint64) * np.uint64(977)
    vec = philox.words(99, 5, 3, 2, blocks)
    for i, b in enumerate(blocks):
        sc = philox.philox4x64(int(b), 5, 3, 2, 99, 0)
        assert [int(v[i]) for v in vec] == [int(s) for s in sc]


def test_uniform52_range_and_exactness():
    w = np.array([0, 1, 2**12 - 1, 2**12, 2**64 - 1, 2**63], dtype=np.uint64)
    u = philox.uniform52(w)
    assert u[0] == 2.0 ** -53 and u[1] == 2.0 ** -53 and u[2] == 2.0 ** -53
    assert u[3] == 1.5 * 2.0 ** -52
    assert u[4] == 1.0 - 2.0 ** -53
    assert u[5] == 0.5 + 2.0 ** -53
    assert np.all((u > 0) & (u < 1))
    # exact: the value times 2^53 is an odd integer
    k = u * 2.0 ** 53
    assert np.all(k == np.floor(k)) and np.all(k % 2 == 1)


def test_uniform24_pair_exact_in_single_precision():
    w = np.array([0, 2**32 - 1, (2**32 - 1) << 32, 123456789 | (987654321 << 32)], dtype=np.uint64)
    lo, hi = philox.uniform24_pair(w)
    assert lo.dtype == np.float32 and hi.dtype == np.float32
    assert lo[0] == np.float32(2.0 ** -33)
    assert lo[1] == np.float32(1.0)            # fl32(2^32 - 1) = 2^32, + 2^-33 rounds to 1
    assert hi[2] == np.float32(1.0) and lo[2] == np.float32(2.0 ** -33)
    # the value is the IEEE single result of the two rounded operations
    x = np.float32(123456789)
    assert lo[3] == np.float32(np.float32(x * np.float32(2.0 ** -32)) + np.float32(2.0 ** -33))


def test_voxel_normals_distribution_and_layout():
    z = philox.voxel_normals(7, 3, philox.STAGE_MOMENTUM, 0, 1 << 18)
    assert abs(z.mean()) < 5.0 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # element 2j and 2j+1 share one word: they are the cos / sin branches of one pair
    ws = philox.words(7, 3, philox.STAGE_MOMENTUM, 0, np.array([5], dtype=np.uint64))
    u1, u2 = philox.uniform24_pair(ws[2])
    r = np.sqrt(-2.0 * np.log(np.float64(u1[0])))
    t = 2.0 * np.pi * np.float64(u2[0])
    assert z[5 * 8 + 4] == pytest.approx(r * np.cos(t), rel=0, abs=1e-15)
    assert z[5 * 8 + 5] == pytest.approx(r * np.sin(t), rel=0, abs=1e-15)
    # odd lengths are a prefix of the full stream
    z2 = philox.voxel_normals(7, 3, philox.STAGE_MOMENTUM, 0, 13)
    assert np.array_equal(z2, z[:13])


def test_streams_are_distinct():
    a = philox.voxel_normals(1, 0, 1, 0, 64)
    b = philox.voxel_normals(1, 1, 1, 0, 64)
    c = philox.voxel_normals(1, 0, 2, 0, 64)
    d = philox.voxel_normals(2, 0, 1, 0, 64)
    for x in (b, c, d):
        assert not np.allclose(a, x)


def test_normal64_law_and_bound():
    # FP64 Box-Muller cosine branch from two words: standard normal, and
    # bounded by sqrt(-2 ln u) at the smallest uniform52 value 2^-53
    w = philox.words(3, 1, 5, 0, np.arange(1 << 15, dtype=np.uint64))
    z = philox.normal64(w[0], w[1])
    assert abs(z.mean()) < 5.0 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert np.max(np.abs(z)) <= np.sqrt(-2.0 * np.log(2.0 ** -53))
    # the definition: u1 from the first word sets the radius, u2 from the second the angle
    u1, u2 = philox.uniform52(w[0][:8]), philox.uniform52(w[1][:8])
    assert np.array_equal(z[:8], np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2))
