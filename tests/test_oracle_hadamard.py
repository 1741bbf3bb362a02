"""Pins for the oracle's Walsh-Hadamard transform (Sec. 2)."""
import os

import numpy as np
import pytest
import scipy.linalg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hadamard_sylvester.txt")


def load_golden():
    mats, cur, n = {}, [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("n="):
            if n is not None:
                mats[n] = np.array(cur, dtype=float)
            n, cur = int(line[2:]), []
        else:
            cur.append([float(v) for v in line.split()])
    mats[n] = np.array(cur, dtype=float)
    return mats


def test_matches_papers_recursion_h2_h4(orc):
    for n, H in load_golden().items():
        assert np.array_equal(orc.hadamard_dense(n), H)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 64, 1024])
def test_dense_equals_scipy(orc, n):
    assert np.array_equal(orc.hadamard_dense(n), scipy.linalg.hadamard(n))


@pytest.mark.parametrize("n", [2, 16, 256])
def test_orthogonality(orc, n):
    H = orc.hadamard_dense(n)
    assert np.array_equal(H.T @ H, n * np.eye(n))
    assert np.array_equal(H, H.T)


@pytest.mark.parametrize("n", [1, 2, 8, 128, 1024])
def test_fast_equals_dense(orc, n):
    rng = np.random.default_rng(n)
    y = rng.standard_normal(n)
    want = scipy.linalg.hadamard(n).astype(float) @ y
    assert np.allclose(orc.fwht(y), want, rtol=1e-13, atol=1e-12 * np.abs(y).sum())


def test_fast_beyond_dense_range_via_kronecker(orc):
    # H_4096 = H_64 (x) H_64 in natural order
    n = 4096
    H64 = scipy.linalg.hadamard(64).astype(float)
    y = np.random.default_rng(1).standard_normal(n)
    want = (H64 @ y.reshape(64, 64) @ H64.T).reshape(-1)
    assert np.allclose(orc.fwht(y), want, rtol=1e-12, atol=1e-11)


def test_involution_and_norm(orc):
    n = 1 << 14
    rng = np.random.default_rng(2)
    y = rng.standard_normal(n)
    z = orc.fwht(y)
    assert np.allclose(orc.fwht(z) / n, y, atol=1e-12)
    # H_n D is orthogonal after normalisation (proof of Thm 1)
    D = rng.choice([-1.0, 1.0], n)
    hd = orc.fwht(D * y) / np.sqrt(n)
    assert abs(np.linalg.norm(hd) / np.linalg.norm(y) - 1.0) < 1e-13


def test_unit_vector_gives_hadamard_column(orc):
    n = 2048
    for j in (0, 1, 5, 1000, 2047):
        e = np.zeros(n)
        e[j] = 1.0
        col = orc.fwht(e)
        i = np.arange(n)
        want = np.where(np.array([bin(v & j).count("1") & 1 for v in i]) == 1, -1.0, 1.0)
        assert np.array_equal(col, want)
