"""Host logic of the Python binding (no GPU): output capacity, padding,
layout marshalling and the decoding of rnnls_info.

The Bernoulli capacity is pinned against the distribution it must cover:
Alg. 1 step 2 keeps each of the n rows with probability r/n, so the row
count is Binomial(n, r/n); the capacity must lie far in its upper tail and
above every count the oracle's sampler draws.
"""
import ctypes

import numpy as np
import pytest
import scipy.stats
import torch

import paper_0812_4547_gb300 as P


@pytest.mark.parametrize("r,n", [(1, 1 << 14), (100, 1 << 14), (4096, 1 << 20), (8192, 1 << 22), (30000, 1 << 16)])
def test_bernoulli_capacity_covers_the_binomial_count(orc, r, n):
    cap = P.bernoulli_capacity(r, n)
    assert scipy.stats.binom.sf(cap, n, r / n) < 1e-8
    counts = [len(orc.sample(seed, 0, n, r, orc.MODE_BERNOULLI, cap=n)) for seed in range(20)]
    assert max(counts) <= cap
    assert cap < r + 7 * np.sqrt(r) + 17  # and not much more than that


def test_bernoulli_capacity_keeps_every_row_when_r_reaches_n():
    assert P.bernoulli_capacity(5000, 4096) == 4096
    assert P.bernoulli_capacity(4096, 4096) == 4096


@pytest.mark.parametrize("n_raw,n", [(1, 1), (2, 2), (3, 4), (4096, 4096), (4097, 8192), ((1 << 20) + 1, 1 << 21)])
def test_padded_n(orc, n_raw, n):
    assert P.padded_n(n_raw) == n == orc.padded_n(n_raw)


def test_colmajor_views_and_copies():
    a = torch.arange(12.0).reshape(3, 4)  # row-major
    c = P.colmajor(a)
    assert c.stride(0) == 1 and torch.equal(c, a)
    assert P.colmajor(c).data_ptr() == c.data_ptr()  # already column-major: a view
    with pytest.raises(ValueError):
        P.colmajor(torch.zeros(3))


@pytest.mark.parametrize("n,d", [(7, 1), (1, 5), (1, 1), (100, 3)])
def test_leading_dimension(n, d):
    t = torch.empty(d, n).t()
    assert P._ld(t) == n
    # a column-major slice of a taller buffer keeps the buffer's leading dimension
    big = torch.empty(d, n + 9).t()[:n]
    assert P._ld(big) == n + 9


def test_info_dict_decodes_the_struct():
    inf = P.rnnls_info(3, 11, 17, 5, 1.5e-12, -2.0, 42.25, 2, 0)
    raw = torch.frombuffer(bytearray(bytes(inf)), dtype=torch.uint8)
    assert raw.numel() == P.INFO_BYTES == ctypes.sizeof(P.rnnls_info) == 48
    got = P.info_dict(raw)
    assert got == {"status": 3, "outer_iters": 11, "inner_iters": 17, "passive_count": 5, "tol": 1.5e-12,
                   "dual_max": -2.0, "objective": 42.25, "accurate_mode": 2, "reserved": 0}
