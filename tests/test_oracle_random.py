"""Pins for the oracle's randomness (Alg. 1 steps 2-4).

The generator is Philox4x64-10 (Salmon et al., SC'11).  numpy ships an
independent implementation of the same generator, which is the pin here.
numpy's Philox advances its counter before producing a block, so block
``ctr`` is numpy's first output when numpy is seeded with ``ctr - 1``.
"""
import math

import numpy as np
import pytest

M64 = (1 << 64) - 1


def numpy_block(ctr, key):
    c = [int(v) for v in ctr]
    # numpy increments the 256-bit counter before use: start one below.
    for i in range(4):
        if c[i] > 0:
            c[i] -= 1
            break
        c[i] = M64
    g = np.random.Philox(counter=np.array(c, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    return g.random_raw(4)


def numpy_word(seed, inst, stream, w):
    return int(numpy_block([w >> 2, stream, 0, 0], [seed, inst])[w & 3])


CASES = [
    ([0, 0, 0, 0], [0, 0]),
    ([1, 0, 0, 0], [7, 3]),
    ([42, 2, 0, 0], [2 ** 63 + 5, 11]),
    ([M64, 1, 0, 0], [123456789, 987654321]),
    ([5, 0, 9, 2 ** 40], [M64, M64]),
]


@pytest.mark.parametrize("ctr,key", CASES)
def test_philox_matches_numpy(orc, ctr, key):
    got = orc.philox4x64_10(np.array(ctr, dtype=np.uint64), np.array(key, dtype=np.uint64))
    want = numpy_block(ctr, key)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("seed,inst", [(0, 0), (3, 17), (2 ** 40 + 1, 2)])
def test_sign_bits_follow_stream0(orc, seed, inst):
    n = 1000
    D = orc.signs(seed, inst, n)
    for i in range(0, n, 37):
        w = numpy_word(seed, inst, 0, i >> 6)
        want = -1 if (w >> (i & 63)) & 1 else 1
        assert D[i] == want
    assert set(np.unique(D)) <= {-1, 1}
    # a fair coin: 1000 draws stay within 5 sigma of 500
    assert abs(int((D < 0).sum()) - n / 2) < 5 * math.sqrt(n / 4)


@pytest.mark.parametrize("n,r", [(1, 3), (2, 5), (4096, 512), (2 ** 22, 300)])
def test_iid_rows_are_top_bits(orc, n, r):
    idx = orc.sample(9, 4, n, r, orc.MODE_IID)
    L = int(math.log2(n))
    assert idx.shape == (r,)
    for k in range(0, r, 7):
        u = numpy_word(9, 4, 2, k)
        want = 0 if L == 0 else u >> (64 - L)
        assert idx[k] == want
    assert idx.min() >= 0 and idx.max() < n


def test_iid_rows_uniform(orc):
    n, r = 64, 64 * 400
    idx = orc.sample(1, 0, n, r, orc.MODE_IID)
    counts = np.bincount(idx, minlength=n)
    chi2 = float(((counts - r / n) ** 2 / (r / n)).sum())
    # chi-square with 63 dof: mean 63, sd ~11.2; 130 is ~6 sd out
    assert chi2 < 130


def test_bernoulli_rows_follow_threshold(orc):
    n, r, L = 1024, 100, 10
    idx = orc.sample(5, 1, n, r, orc.MODE_BERNOULLI)
    thresh = r << (64 - L)
    want = [i for i in range(n) if numpy_word(5, 1, 1, i) < thresh]
    assert idx.tolist() == want
    assert np.all(np.diff(idx) > 0)


def test_bernoulli_count_binomial(orc):
    n, r = 4096, 256
    counts = np.array([len(orc.sample(s, 0, n, r, orc.MODE_BERNOULLI)) for s in range(200)])
    p = r / n
    mean, var = n * p, n * p * (1 - p)
    assert abs(counts.mean() - mean) < 5 * math.sqrt(var / len(counts))
    assert 0.5 * var < counts.var() < 1.6 * var


def test_bernoulli_r_ge_n_keeps_every_row(orc):
    idx = orc.sample(0, 0, 256, 256, orc.MODE_BERNOULLI)
    assert idx.tolist() == list(range(256))
    assert orc.scale(256, 300, orc.MODE_BERNOULLI) == pytest.approx(1 / 16)
    assert orc.scale(256, 64, orc.MODE_BERNOULLI) == pytest.approx(1 / 8)
    assert orc.scale(256, 300, orc.MODE_IID) == pytest.approx(1 / math.sqrt(300))


def test_streams_are_independent_of_each_other(orc):
    # signs and sampling use different stream words of the same key
    a = numpy_word(0, 0, 0, 0)
    b = numpy_word(0, 0, 1, 0)
    c = numpy_word(0, 0, 2, 0)
    assert len({a, b, c}) == 3
    assert not np.array_equal(orc.sample(0, 0, 1 << 20, 64), orc.sample(0, 1, 1 << 20, 64))
