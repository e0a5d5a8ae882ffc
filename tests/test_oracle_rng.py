"""Pins of the oracle's random draws against things other than the oracle itself.

* Philox4x32-10 against the published known-answer vectors (tests/golden/philox4x32_kat.txt).
* The same round structure at 64-bit width (Philox4x64-10) against NumPy's own Philox
  bit generator, which implements that variant.
* The uniform, normal and index maps against their laws (exact end points, moments,
  Kolmogorov-Smirnov, chi-square), i.e. against the uniform sampling law xi^u_j = 1/n
  of Eq. (unique) and the N(0,1) entries of the reparameterised matrices.
"""
import os

import numpy as np
import pytest
import scipy.stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox4x32_known_answers(ctr, key, expect):
    assert list(oracle.philox4x32(ctr, key)) == expect


def test_philox4x64_matches_numpy():
    # NumPy's Philox is Philox4x64-10; it advances its 256-bit counter before each block.
    rng = np.random.default_rng(11)
    for _ in range(20):
        key = rng.integers(0, 2**63, size=2, dtype=np.uint64)
        ctr = rng.integers(0, 2**63, size=4, dtype=np.uint64)
        bg = np.random.Philox(key=key, counter=ctr)
        raw = bg.random_raw(8)
        c = [int(x) for x in ctr]
        for blk in range(2):
            v = c[0] + blk + 1
            c1 = [v % 2**64, c[1] + (v >> 64), c[2], c[3]]
            out = oracle.philox4x64(c1, key)
            assert list(out) == list(raw[4 * blk:4 * blk + 4])


def test_uniform_map_endpoints_and_exactness():
    assert oracle.uniform(0) == 2.0**-33
    assert oracle.uniform(2**32 - 1) == 1.0 - 2.0**-33
    for w in (1, 12345, 2**31, 2**32 - 2):
        assert oracle.uniform(w) == (w + 0.5) / 2.0**32


def test_normal_law():
    # 4 normals per Philox call (two Box-Muller pairs); sample over rows i and inner k.
    z = np.array([oracle.normal(5, 0, 3, 17, i, k) for i in range(64) for k in range(600)])
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / z.size)
    ks = scipy.stats.kstest(z, "norm")
    assert ks.pvalue > 1e-4
    # the four normals of one call (rows 4q..4q+3) are pairwise uncorrelated
    zz = z.reshape(16, 4, 600).transpose(1, 0, 2).reshape(4, -1)
    c = np.corrcoef(zz)
    assert np.max(np.abs(c - np.eye(4))) < 5 / np.sqrt(zz.shape[1])


def test_normal_is_a_function_of_its_coordinates():
    a = oracle.normal(0, 0, 2, 5, 7, 11)
    assert a == oracle.normal(0, 0, 2, 5, 7, 11)
    others = [oracle.normal(1, 0, 2, 5, 7, 11), oracle.normal(0, 1, 2, 5, 7, 11),
              oracle.normal(0, 0, 3, 5, 7, 11), oracle.normal(0, 0, 2, 6, 7, 11),
              oracle.normal(0, 0, 2, 5, 6, 11), oracle.normal(0, 0, 2, 5, 7, 12),
              oracle.normal(0, 0, 2, 5 + 2**32, 7, 11)]
    assert all(o != a for o in others)


def test_index_law_chi_square():
    n = 37
    draws = np.array([oracle.index(2, 0, 1, s, t, n) for s in range(400) for t in range(150)])
    assert draws.min() >= 0 and draws.max() < n
    counts = np.bincount(draws, minlength=n)
    chi = scipy.stats.chisquare(counts)
    assert chi.pvalue > 1e-4


def test_index_edge_cases():
    assert all(oracle.index(9, 3, 0, s, t, 1) == 0 for s in range(20) for t in range(8))
    big = 2**31 - 1
    v = [oracle.index(1, 0, 5, s, t, big) for s in range(50) for t in range(4)]
    assert min(v) >= 0 and max(v) < big
    # even and odd slots of one call use different halves of the block
    assert oracle.index(2, 0, 0, 0, 0, 2**40) != oracle.index(2, 0, 0, 0, 1, 2**40)


def test_index_from_block_words():
    # slot t takes the 64-bit word (w1:w0) for even t and (w3:w2) for odd t of the block
    # with counter (t/2, 0xFFFFFFFF, s_lo, s_hi << 8 | l), and maps it by floor(word * n / 2^64).
    n, l, s = 1000003, 4, (7 << 32) | 99
    for t in range(6):
        w = oracle.philox4x32([t >> 1, 0xFFFFFFFF, s & 0xFFFFFFFF, ((s >> 32) << 8) | l], [2, 5])
        word = (int(w[3]) << 32 | int(w[2])) if t & 1 else (int(w[1]) << 32 | int(w[0]))
        assert oracle.index(2, 5, l, s, t, n) == (word * n) >> 64
