"""The seeded input recipe (stand-ins for the paper's term-document data,
Sec. 4.1) against its stated distributions: density, value law and column
scale of the term-document matrices, the exact zero count of the planted
solutions, the noise level of the targets, and the ranges of the uneven
batch.  Statistical checks use bounds several standard errors wide.
"""
import math

import numpy as np
import pytest

import workloads


def test_termdoc_density_values_and_column_scale():
    n, cols = 200_000, 64
    A = workloads.termdoc_matrix(n, cols, np.random.default_rng(1))
    assert A.dtype == np.float32 and A.flags.f_contiguous and np.all(A >= 0)
    nz = A != 0
    p = nz.mean()
    assert abs(p - 0.02) < 4 * math.sqrt(0.02 * 0.98 / A.size)
    # a row is empty with probability 0.98^64 (about 27 %)
    empty = 1.0 - nz.any(axis=1).mean()
    assert abs(empty - 0.98 ** cols) < 0.01
    # non-zeros of column j: LogNormal(0, 1) * (j + 1)^-1.1, so log(value) + 1.1 log(j + 1) ~ N(0, 1)
    for j in (0, 7, 63):
        v = A[nz[:, j], j].astype(np.float64)
        z = np.log(v) + 1.1 * math.log(j + 1)
        assert abs(z.mean()) < 4 / math.sqrt(len(z))
        assert abs(z.std() - 1.0) < 0.1


def test_planted_x_has_the_exact_zero_count():
    rng = np.random.default_rng(2)
    for d, nz in ((20, 10), (64, 32), (100, 30), (7, 0), (5, 5)):
        x = workloads.planted_x(d, nz, rng)
        assert np.count_nonzero(x == 0.0) == nz
        assert np.all((x >= 0) & (x <= 2))


def test_noisy_target_noise_level():
    rng = np.random.default_rng(3)
    A = workloads.termdoc_matrix(100_000, 10, rng)
    x = workloads.planted_x(10, 5, rng)
    b = workloads.noisy_target(A, x, rng, noise_rel=0.05)
    clean = A.astype(np.float64) @ x
    sigma = 0.05 * np.linalg.norm(clean) / math.sqrt(len(b))
    assert np.std(b - clean) == pytest.approx(sigma, rel=0.02)
    b_abs = workloads.noisy_target(A, x, rng, noise_abs=0.01)
    assert np.std(b_abs - clean) == pytest.approx(0.01, rel=0.02)


def test_problem_shapes_and_types():
    p = workloads.problem(1)
    assert p.A.shape == (4096, 20) and p.A.dtype == np.float64 and p.r == 512
    assert np.count_nonzero(p.x_true == 0) == 10
    p = workloads.problem(2, n=1 << 12)
    assert p.A.shape == (1 << 12, 64) and p.A.dtype == np.float32 and p.b.dtype == np.float32 and p.r == 4096
    assert np.count_nonzero(p.x_true == 0) == 32
    A, B, X, r = workloads.multi_rhs(n=1 << 12, nrhs=6)
    assert A.shape == (1 << 12, 100) and B.shape == (1 << 12, 6) and X.shape == (100, 6) and r == 4096
    zeros = (X == 0).sum(axis=0)
    assert np.all((zeros >= 30) & (zeros <= 80))


def test_batch_shapes_ranges():
    shapes = workloads.batch_shapes()
    assert len(shapes) == 512
    for n_raw, d, r in shapes:
        assert (1 << 14) <= n_raw < (1 << 20)
        assert 16 <= d <= 200
        n = workloads.next_pow2(n_raw)
        target = 8 * (d + 1) * math.log(n)
        assert r >= target and r < 2 * target and r & (r - 1) == 0
        assert 2048 <= r <= 32768
    ds = np.array([d for _, d, _ in shapes])
    assert ds.min() <= 20 and ds.max() >= 196  # the whole range is drawn
    assert workloads.batch_shapes() == shapes  # seeded


def test_same_seed_same_bytes():
    a = workloads.problem(2, n=5000, seed=9)
    b = workloads.problem(2, n=5000, seed=9)
    assert np.array_equal(a.A, b.A) and np.array_equal(a.b, b.b)
    c = workloads.problem(2, n=5000, seed=10)
    assert not np.array_equal(a.A, c.A)
