"""Pins for the oracle's random sketching matrix (Algorithms 1 and 2, step 2).

The method needs G with independent N(0, 1) entries (section 4.1; Lemma 4.4 and
Theorem 4.5 assume exactly that).  These tests check the oracle's generator
against what that fixes -- the standard normal law, independence, the uniform
grid, and the accuracy of our own log / sin / cos against libm -- rather than
against itself.
"""
import math

import numpy as np
import pytest

import oracle as O


def test_uniform_grid_and_range():
    xs = [0, 1, 511, 512, 0x7FFFFFFF, 0x80000000, 0xFFFFFE00, 0xFFFFFFFF]
    for x in xs:
        u = O.uniform(x)
        k = u * 2.0 ** 24
        assert 0.0 < u < 1.0
        assert k == int(k) and int(k) % 2 == 1          # odd multiple of 2^-24
        assert int(k) == 2 * (x >> 9) + 1
    assert O.uniform(0) == 2.0 ** -24
    assert O.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24


def test_own_log_matches_libm():
    rng = np.random.Generator(np.random.PCG64(5))
    xs = np.concatenate([rng.integers(0, 2 ** 32, 20000, dtype=np.uint64),
                         np.array([0, 1, 2 ** 31, 2 ** 32 - 1], dtype=np.uint64)])
    worst = 0.0
    for x in xs:
        u = O.uniform(int(x))
        got = O.logf(u)
        ref = math.log(u)
        ulp = float(np.spacing(np.float32(abs(ref)))) if ref != 0 else 1e-45
        worst = max(worst, abs(got - ref) / ulp)
    assert worst <= 2.0, worst


def test_own_sincos_matches_libm():
    rng = np.random.Generator(np.random.PCG64(6))
    xs = np.concatenate([rng.integers(0, 2 ** 32, 20000, dtype=np.uint64),
                         np.array([0, 2 ** 30, 2 ** 31, 3 * 2 ** 30, 2 ** 32 - 1], dtype=np.uint64)])
    worst = 0.0
    for x in xs:
        u = O.uniform(int(x))
        s, c = O.sincos2pi(u)
        worst = max(worst, abs(s - math.sin(2 * math.pi * u)), abs(c - math.cos(2 * math.pi * u)))
    assert worst <= 3e-7, worst


def test_box_muller_assembly_against_definition():
    # z(4q+0) = sqrt(-2 ln u0) cos(2 pi u1), z(4q+1) = ... sin, z(4q+2/3) from words 2, 3.
    seed, tag, i = 12345, 0, 7
    for q in (0, 1, 1000, 2 ** 20 + 3):
        w = O.philox4x32_10((q & 0xFFFFFFFF, q >> 32, i, tag), (seed & 0xFFFFFFFF, seed >> 32))
        u = [O.uniform(v) for v in w]
        ref = [math.sqrt(-2 * math.log(u[0])) * math.cos(2 * math.pi * u[1]),
               math.sqrt(-2 * math.log(u[0])) * math.sin(2 * math.pi * u[1]),
               math.sqrt(-2 * math.log(u[2])) * math.cos(2 * math.pi * u[3]),
               math.sqrt(-2 * math.log(u[2])) * math.sin(2 * math.pi * u[3])]
        got = [O.normal_at(seed, tag, i, 4 * q + k) for k in range(4)]
        for g, r in zip(got, ref):
            assert abs(g - r) <= 4e-6 * max(1.0, abs(r)), (q, got, ref)


def test_philox_bijective_and_avalanche():
    key = (0xDEADBEEF, 0x01234567)
    outs = set()
    flips = []
    rng = np.random.Generator(np.random.PCG64(9))
    for t in range(3000):
        ctr = tuple(int(v) for v in rng.integers(0, 2 ** 32, 4, dtype=np.uint64))
        o = O.philox4x32_10(ctr, key)
        outs.add(o)
        bit = t % 128
        c2 = list(ctr)
        c2[bit // 32] ^= 1 << (bit % 32)
        o2 = O.philox4x32_10(c2, key)
        flips.append(sum(bin(a ^ b).count("1") for a, b in zip(o, o2)))
    assert len(outs) == 3000
    mean = float(np.mean(flips))
    assert abs(mean - 64.0) < 1.0, mean            # ~half of 128 output bits flip


def test_normals_moments_and_ks():
    from scipy import stats
    z = O.normals(2024, 0, 0, 0, 500, 2000).astype(np.float64).ravel()
    n = z.size
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(stats.skew(z)) < 5 * math.sqrt(6.0 / n)
    assert abs(stats.kurtosis(z)) < 5 * math.sqrt(24.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4


def test_normals_independent_across_index_and_seed():
    a = O.normals(1, 0, 0, 0, 400, 1000).astype(np.float64)
    b = O.normals(2, 0, 0, 0, 400, 1000).astype(np.float64)
    c = O.normals(1, 1, 0, 0, 400, 1000).astype(np.float64)
    n = a.size
    lim = 5 / math.sqrt(n)
    assert abs(np.corrcoef(a.ravel(), b.ravel())[0, 1]) < lim          # seeds
    assert abs(np.corrcoef(a.ravel(), c.ravel())[0, 1]) < lim          # tags
    assert abs(np.corrcoef(a[:, :-1].ravel(), a[:, 1:].ravel())[0, 1]) < lim   # neighbours in j
    assert abs(np.corrcoef(a[:-1].ravel(), a[1:].ravel())[0, 1]) < lim         # neighbours in i
    assert abs(np.corrcoef(a[:, 0::4].ravel(), a[:, 1::4].ravel())[0, 1]) < 5 / math.sqrt(n / 4)


def test_blocks_are_windows_of_one_matrix():
    full = O.normals(77, 0, 0, 0, 16, 40)
    part = O.normals(77, 0, 5, 13, 7, 19)
    assert np.array_equal(full[5:12, 13:32], part)
    assert O.normal_at(77, 0, 5, 13) == full[5, 13]


def test_sketch_entries_are_normals_on_grid():
    z = O.normals(3, 0, 0, 0, 64, 256).astype(np.float64)
    g = O.sketch_block(3, 0, 0, 64, 256)
    q = g * 4096.0
    assert np.array_equal(q, np.round(q))
    assert np.max(np.abs(g - z)) <= 2.0 ** -13
    assert np.max(np.abs(q)) <= 32767


@pytest.mark.parametrize("j", [0, 1, 2, 3, 4, 2 ** 32 + 5])
def test_large_column_index(j):
    # columns beyond 2^32 use the second counter word; still a normal draw
    v = O.normal_at(11, 0, 3, j)
    assert math.isfinite(v) and abs(v) < 8
