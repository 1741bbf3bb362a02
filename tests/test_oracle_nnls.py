"""Pins for the oracle's Lawson-Hanson NNLS (Alg. 1 step 5, Def. 1).

Pins: scipy.optimize.nnls (an independent active-set code), brute force over
all 2^d passive sets, the KKT conditions, the unconstrained special case
(numpy lstsq) and closed-form degenerate cases.
"""
import itertools

import numpy as np
import pytest
import scipy.optimize

import workloads


def kkt(S, s, x, tol_rel=1e-9):
    g = S.T @ (S @ x - s)  # gradient / 2
    scale = np.linalg.norm(S, 1) * np.linalg.norm(s) + 1e-300
    assert np.all(x >= 0)
    assert np.all(g >= -tol_rel * scale)
    assert np.all(np.abs(g[x > 0]) <= tol_rel * scale)
    assert np.all(np.abs(x * g) <= 1e-10 * scale * (np.abs(x).max() + 1e-300))


def brute_force_nnls(S, s):
    """Unique optimum by enumeration: the passive set whose LS solution is
    positive and satisfies dual feasibility."""
    d = S.shape[1]
    best = None
    for k in range(d + 1):
        for P in itertools.combinations(range(d), k):
            x = np.zeros(d)
            if P:
                sol, *_ = np.linalg.lstsq(S[:, P], s, rcond=None)
                if np.any(sol <= 0):
                    continue
                x[list(P)] = sol
            g = S.T @ (S @ x - s)
            if np.all(g >= -1e-9 * np.linalg.norm(S.T @ s)):
                obj = np.linalg.norm(S @ x - s)
                if best is None or obj < best[0] - 1e-12:
                    best = (obj, x)
    return best[1]


@pytest.mark.parametrize("seed", range(6))
def test_matches_scipy_nnls(orc, seed):
    rng = np.random.default_rng(seed)
    m, d = 200, 15
    S = rng.standard_normal((m, d))
    s = rng.standard_normal(m) + S @ np.maximum(rng.standard_normal(d), 0)
    x, info = orc.nnls(S, s)
    xs, _ = scipy.optimize.nnls(S, s)
    assert info["status"] == orc.OK
    assert np.linalg.norm(x - xs) <= 1e-10 * max(np.linalg.norm(xs), 1.0)
    kkt(S, s, x)


@pytest.mark.parametrize("seed,d", [(0, 4), (1, 6), (2, 8), (3, 10), (4, 10)])
def test_active_set_matches_brute_force(orc, seed, d):
    rng = np.random.default_rng(100 + seed)
    S = rng.standard_normal((40, d))
    s = rng.standard_normal(40)
    x, info = orc.nnls(S, s)
    xb = brute_force_nnls(S, s)
    assert np.array_equal(x > 0, xb > 0)
    assert np.allclose(x, xb, atol=1e-10)


def test_unconstrained_special_case(orc):
    rng = np.random.default_rng(11)
    S = rng.random((100, 6)) + 0.1
    xt = rng.uniform(0.5, 2.0, 6)
    s = S @ xt + 0.001 * rng.standard_normal(100)
    xl, *_ = np.linalg.lstsq(S, s, rcond=None)
    assert np.all(xl > 0)
    x, _ = orc.nnls(S, s)
    assert np.allclose(x, xl, rtol=1e-11)


def test_gram_form(orc):
    rng = np.random.default_rng(12)
    S = rng.standard_normal((50, 7))
    s = rng.standard_normal(50)
    Q, q, ss = orc.gram(S, s)
    assert np.allclose(Q, S.T @ S, rtol=1e-14)
    assert np.allclose(q, S.T @ s, rtol=1e-14)
    assert ss == pytest.approx(s @ s, rel=1e-14)


def test_degenerate_cases(orc):
    rng = np.random.default_rng(13)
    S = rng.random((30, 5))
    # zero target: x = 0
    x, info = orc.nnls(S, np.zeros(30))
    assert np.array_equal(x, np.zeros(5)) and info["passive_count"] == 0
    # target anti-correlated with every column: x = 0
    x, _ = orc.nnls(S, -S.sum(axis=1))
    assert np.array_equal(x, np.zeros(5))
    # one column
    x, _ = orc.nnls(S[:, :1], S[:, 0] * 3.0)
    assert x[0] == pytest.approx(3.0, rel=1e-13)


def test_rank_deficient_duplicate_column(orc):
    rng = np.random.default_rng(14)
    S = rng.random((60, 4))
    S = np.hstack([S, S[:, :1]])  # column 4 duplicates column 0
    s = S[:, :4] @ np.array([1.0, 0.5, 0.0, 2.0]) + 0.01 * rng.standard_normal(60)
    x, info = orc.nnls(S, s)
    xs, _ = scipy.optimize.nnls(S, s)
    assert info["status"] == orc.OK
    assert np.linalg.norm(S @ x - s) == pytest.approx(np.linalg.norm(S @ xs - s), rel=1e-10)


def test_iteration_cap(orc):
    rng = np.random.default_rng(15)
    S = rng.random((80, 10)) + 0.05
    s = S @ rng.uniform(0.5, 1.0, 10)
    Q, q, _ = orc.gram(S, s)
    tol = orc.lh_tol(S, s)
    x, info = orc.nnls_lh(Q, q, tol, max_outer=1)
    assert info["status"] == orc.EMAXITER
    x, info = orc.nnls_lh(Q, q, tol)
    assert info["status"] == orc.OK and info["passive_count"] == 10


def test_randomized_nnls_ratio_at_least_one(orc):
    # Theorem 1's ratio ||A x~ - b||^2 / ||A x_opt - b||^2 is >= 1 (x_opt is optimal)
    p = workloads.problem(2, n=1 << 13, d=16, r=512)
    xo, io = orc.exact_nnls(p.A, p.b)
    assert io["status"] == orc.OK
    kkt(p.A.astype(float), p.b.astype(float), xo, tol_rel=1e-8)
    opt = orc.residual_sq(p.A, p.b, xo)
    ratios = []
    for seed in range(3):
        xt, it, _ = orc.randomized_nnls(p.A, p.b, p.r, seed)
        assert it["status"] == orc.OK
        ratios.append(orc.residual_sq(p.A, p.b, xt) / opt)
    assert min(ratios) >= 1.0 - 1e-12
    assert max(ratios) < 1.5


def test_keep_all_rows_recovers_exact_solution(orc):
    # Bernoulli mode with r >= n: S H D is orthogonal, so x~ = x_opt
    p = workloads.problem(1, n=1000, d=8)
    xo, _ = orc.exact_nnls(p.A, p.b)
    xt, _, _ = orc.randomized_nnls(p.A, p.b, 4096, seed=3, mode=orc.MODE_BERNOULLI)
    assert np.allclose(xt, xo, rtol=1e-9, atol=1e-12)


def test_residual_sq(orc):
    rng = np.random.default_rng(16)
    A = rng.random((77, 3))
    b = rng.random(77)
    x = rng.random(3)
    assert orc.residual_sq(A, b, x) == pytest.approx(np.sum((A @ x - b) ** 2), rel=1e-13)


def test_tie_break_smallest_index(orc):
    # Column 3 duplicates column 1, so their duals tie exactly at every step:
    # the rule "ties go to the smallest index" admits column 1; column 3 is
    # then numerically dependent and stays at zero.
    rng = np.random.default_rng(17)
    S = rng.random((50, 3)) + 0.1
    S = np.hstack([S, S[:, 1:2]])
    s = S[:, :3] @ np.array([0.2, 1.0, 0.3])
    x, info = orc.nnls(S, s)
    assert info["status"] == orc.OK
    assert x[1] > 0 and x[3] == 0.0


def test_rejection_rule_keeps_solver_finite(orc):
    # With a negative tolerance every column with w_j in (tol, 0] is tried;
    # its passive solve gives z_j <= 0 and must be rejected (the NNLS
    # routine's rule), otherwise the method cycles on it until the cap.
    rng = np.random.default_rng(18)
    S = rng.standard_normal((60, 8))
    s = rng.standard_normal(60)
    Q, q, _ = orc.gram(S, s)
    x0, i0 = orc.nnls_lh(Q, q, orc.lh_tol(S, s))
    assert 0 < i0["passive_count"] < 8
    x1, i1 = orc.nnls_lh(Q, q, -1e6)
    assert i1["status"] == orc.OK
    assert np.allclose(x1, x0, atol=1e-12)


@pytest.mark.parametrize("seed", range(40))
def test_objective_never_increases(orc, seed):
    # Lawson-Hanson is a descent method: each interpolation step
    # x <- x + alpha (z - x) and each passive solve lowers x'Qx/2 - q'x.
    # Nearly low-rank columns make later admissions push earlier variables
    # negative, so most of these cases run the interpolation step.
    rng = np.random.default_rng(300 + seed)
    S = rng.standard_normal((40, 3)) @ rng.standard_normal((3, 15)) + 0.1 * rng.standard_normal((40, 15))
    s = rng.standard_normal(40)
    Q, q, _ = orc.gram(S, s)
    x, info = orc.nnls_lh(Q, q, orc.lh_tol(S, s), trace=True)
    tr = info["trace"]
    assert info["status"] == orc.OK
    scale = np.abs(tr).max() + 1e-300
    assert np.all(np.diff(tr) <= 1e-12 * scale)
    xs, _ = scipy.optimize.nnls(S, s)
    assert np.linalg.norm(S @ x - s) <= np.linalg.norm(S @ xs - s) * (1 + 1e-10)
