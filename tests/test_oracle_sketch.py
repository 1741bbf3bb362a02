"""Pins for the oracle's sketch H~ D [A b] (Alg. 1 steps 1-5).

The strongest pin writes the sketch out as a dense product with scipy's
Hadamard matrix and with D and the sampled rows taken from numpy's Philox,
so a wrong sign, row, scale or padding in the oracle fails it.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from tests.test_oracle_random import numpy_word


def dense_sketch(A, b, r, seed, inst, mode):
    n_raw, d = A.shape
    n = 1
    while n < n_raw:
        n <<= 1
    L = int(math.log2(n))
    X = np.zeros((n, d + 1))
    X[:n_raw, :d] = A
    X[:n_raw, d] = b
    D = np.array([-1.0 if (numpy_word(seed, inst, 0, i >> 6) >> (i & 63)) & 1 else 1.0 for i in range(n)])
    if mode == 0:
        idx = np.array([0 if L == 0 else numpy_word(seed, inst, 2, k) >> (64 - L) for k in range(r)], dtype=np.int64)
        sc = 1 / math.sqrt(r)
    else:
        if r >= n:
            idx = np.arange(n)
            sc = 1 / math.sqrt(n)
        else:
            idx = np.array([i for i in range(n) if numpy_word(seed, inst, 1, i) < (r << (64 - L))], dtype=np.int64)
            sc = 1 / math.sqrt(r)
    H = scipy.linalg.hadamard(n).astype(float)
    SX = sc * (H[idx] @ (D[:, None] * X))
    return SX[:, :d], SX[:, d], idx


@pytest.mark.parametrize("n_raw,d,r,mode", [
    (1, 1, 1, 0), (2, 1, 3, 0), (5, 2, 4, 0), (64, 3, 16, 0), (100, 4, 40, 0), (1000, 3, 200, 0),
    (64, 3, 16, 1), (100, 4, 40, 1), (33, 2, 64, 1), (1000, 3, 200, 1),
])
def test_sketch_equals_dense_definition(orc, n_raw, d, r, mode):
    rng = np.random.default_rng(n_raw * 31 + d)
    A = rng.standard_normal((n_raw, d))
    b = rng.standard_normal(n_raw)
    SA, Sb, idx = orc.sketch(A, b, r, seed=11, instance=3, mode=mode)
    SA2, Sb2, idx2 = dense_sketch(A, b, r, 11, 3, mode)
    assert np.array_equal(idx, idx2)
    assert np.allclose(SA, SA2, rtol=1e-12, atol=1e-12)
    assert np.allclose(Sb, Sb2, rtol=1e-12, atol=1e-12)


def test_sketch_fast_path_via_kronecker(orc):
    # n = 4096 > 1024 takes the iterative transform: check through H_64 (x) H_64
    n, d, r = 4096, 2, 50
    rng = np.random.default_rng(7)
    A = rng.random((n, d))
    b = rng.random(n)
    SA, Sb, idx = orc.sketch(A, b, r, seed=0)
    H64 = scipy.linalg.hadamard(64).astype(float)
    D = orc.signs(0, 0, n).astype(float)
    for j in range(d + 1):
        x = (A[:, j] if j < d else b) * D
        y = (H64 @ x.reshape(64, 64) @ H64.T).reshape(-1)
        got = SA[:, j] if j < d else Sb
        assert np.allclose(got, y[idx] / math.sqrt(r), rtol=1e-12, atol=1e-12)


def test_padding_equals_explicit_zero_rows(orc):
    rng = np.random.default_rng(3)
    A = rng.random((1500, 3))
    b = rng.random(1500)
    Ap = np.vstack([A, np.zeros((2048 - 1500, 3))])
    bp = np.concatenate([b, np.zeros(2048 - 1500)])
    s1 = orc.sketch(A, b, 77, seed=5)
    s2 = orc.sketch(Ap, bp, 77, seed=5)
    for u, v in zip(s1, s2):
        assert np.array_equal(u, v)


def test_linearity_and_column_independence(orc):
    rng = np.random.default_rng(4)
    A1, A2 = rng.random((3000, 4)), rng.random((3000, 4))
    b1, b2 = rng.random(3000), rng.random(3000)
    s1 = orc.sketch(A1, b1, 100, seed=2)
    s2 = orc.sketch(A2, b2, 100, seed=2)
    s3 = orc.sketch(2 * A1 - 3 * A2, 2 * b1 - 3 * b2, 100, seed=2)
    assert np.allclose(s3[0], 2 * s1[0] - 3 * s2[0], atol=1e-11)
    assert np.allclose(s3[1], 2 * s1[1] - 3 * s2[1], atol=1e-11)
    # a column's sketch does not depend on the other columns
    s4 = orc.sketch(A1[:, :2], b1, 100, seed=2)
    assert np.array_equal(s4[0], s1[0][:, :2])
    assert np.array_equal(s4[1], s1[1])


def test_entry_from_definition_matches(orc):
    rng = np.random.default_rng(5)
    n = 5000
    A = rng.random((n, 2))
    b = rng.random(n)
    SA, Sb, idx = orc.sketch(A, b, 64, seed=9, instance=1)
    sc = 1 / math.sqrt(64)
    for k in (0, 13, 63):
        assert orc.sketch_entry(A[:, 1], 9, 1, int(idx[k]), sc) == pytest.approx(SA[k, 1], rel=1e-12, abs=1e-12)
        assert orc.sketch_entry(b, 9, 1, int(idx[k]), sc) == pytest.approx(Sb[k], rel=1e-12, abs=1e-12)


def test_keep_all_rows_preserves_every_residual(orc):
    # Bernoulli with r >= n keeps every row with factor 1/sqrt(n): S H D is orthogonal
    rng = np.random.default_rng(6)
    A = rng.random((200, 5))
    b = rng.random(200)
    SA, Sb, idx = orc.sketch(A, b, 256, seed=1, mode=orc.MODE_BERNOULLI)
    assert len(idx) == 256
    for _ in range(5):
        x = rng.standard_normal(5)
        assert np.linalg.norm(SA @ x - Sb) == pytest.approx(np.linalg.norm(A @ x - b), rel=1e-12)


def test_norm_estimate_unbiased(orc):
    # Lemma 1's estimator: E ||S H D Phi y||^2 = ||Phi y||^2 over the randomness
    rng = np.random.default_rng(8)
    n, d = 512, 3
    A = rng.random((n, d))
    b = rng.random(n)
    y = np.array([0.3, -0.2, 0.5])
    target = np.linalg.norm(A @ y - b) ** 2
    ests = []
    for s in range(300):
        SA, Sb, _ = orc.sketch(A, b, 32, seed=s)
        ests.append(np.linalg.norm(SA @ y - Sb) ** 2)
    ests = np.array(ests)
    assert abs(ests.mean() - target) < 5 * ests.std() / math.sqrt(len(ests))


def test_norm_estimate_relative_error_lemma1(orc):
    # Lemma 1: with enough rows every y has | ||Phi y||^2 - ||S Phi y||^2 | <= eps ||Phi y||^2
    # (w.p. >= 2/3).  At r = 2048, d + 1 = 4, n = 2^14 the relative error is small.
    rng = np.random.default_rng(9)
    n = 1 << 14
    A = rng.random((n, 3))
    b = rng.random(n)
    ok = 0
    for s in range(6):
        SA, Sb, _ = orc.sketch(A, b, 2048, seed=s)
        worst = 0.0
        for _ in range(20):
            y = rng.standard_normal(3)
            t = np.linalg.norm(A @ y - b) ** 2
            e = np.linalg.norm(SA @ y - Sb) ** 2
            worst = max(worst, abs(t - e) / t)
        ok += worst < 0.25
    assert ok >= 4


def test_lemma2_leverage_flattening(orc):
    # Lemma 2: rows of H_n D U have squared norm <= 4.2 d log2(n) / n w.p. >= 0.9
    rng = np.random.default_rng(10)
    n, d = 1024, 4
    U, _ = np.linalg.qr(rng.standard_normal((n, d)) * (1 + 50 * (np.arange(n) < 8))[:, None])
    H = scipy.linalg.hadamard(n).astype(float) / math.sqrt(n)
    bound = 4.2 * d * math.log2(n) / n
    passes = 0
    for s in range(20):
        D = orc.signs(s, 0, n).astype(float)
        rows = np.sum((H @ (D[:, None] * U)) ** 2, axis=1)
        passes += rows.max() <= bound
    assert passes >= 18
