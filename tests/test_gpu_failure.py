"""Failure paths of the GPU library, each made on the host (no fault, no hang).

Non-finite data must come back as a status, never as a quiet wrong answer:
a NaN or an infinity in SA or Sb, or in A or b upstream of the sketch, ends
that solve with RNNLS_ENONFINITE and x = 0; the other problems of a batched
or multi-target call are untouched (their x still equal to the oracle's on
their own data); and the context stays usable for the next call.  A
rank-deficient sketch (a repeated column) is not an error: Lawson-Hanson
leaves the dependent copy at zero and reaches the same objective as the
oracle, which is the unique part of the answer when the argmin is not.
"""
import numpy as np
import pytest

from tests.gpu_util import dev_colmajor, dev_vec, host

pytestmark = pytest.mark.gpu

ENONFINITE = 3
TOL_X = 1e-6


@pytest.fixture(scope="module")
def ctx():
    import paper_0812_4547_gb300 as P

    c = P.Context(0)
    yield c
    c.close()


def _good(m, d, seed):
    rng = np.random.default_rng(seed)
    S = rng.standard_normal((m, d)).astype(np.float32)
    s = (S.astype(np.float64) @ np.maximum(rng.standard_normal(d), 0) + 0.1 * rng.standard_normal(m)).astype(np.float32)
    return S, s


def _matches_oracle(orc, x, info, S, s):
    xo, io = orc.nnls(S.astype(np.float64), s.astype(np.float64))
    assert info["status"] == io["status"] == 0, (info, io)
    assert np.array_equal(x > 0, xo > 0)
    assert np.linalg.norm(x - xo) <= TOL_X * max(np.linalg.norm(xo), 1e-300)


def _reported(x, info):
    assert info["status"] == ENONFINITE, info
    assert np.all(x == 0.0)


@pytest.mark.parametrize("where", ["SA", "Sb"])
@pytest.mark.parametrize("value", [np.nan, np.inf, -np.inf])
def test_nonfinite_sketch_is_reported_and_context_survives(ctx, orc, where, value):
    import paper_0812_4547_gb300 as P

    S, s = _good(300, 12, 1)
    Sbad, sbad = S.copy(), s.copy()
    if where == "SA":
        Sbad[17, 5] = value
    else:
        sbad[40] = value
    x, info = ctx.solve(dev_colmajor(Sbad), dev_vec(sbad))
    _reported(host(x), P.info_dict(info))
    # the same context, the next call: a plain solve
    x, info = ctx.solve(dev_colmajor(S), dev_vec(s))
    _matches_oracle(orc, host(x), P.info_dict(info), S, s)


def test_infinite_input_through_the_sketch(ctx, orc):
    """An infinity in A reaches every sampled row of its column (each sketch row
    sums over all rows of A) and the solve reports it."""
    import paper_0812_4547_gb300 as P

    rng = np.random.default_rng(2)
    n, d, r = 20000, 4, 200
    A = rng.random((n, d)).astype(np.float32)
    b = rng.random(n).astype(np.float32)
    A[12345, 1] = np.inf
    SA, Sb, _, rows = ctx.sketch(dev_colmajor(A), dev_vec(b), r, seed=3)
    SAh = host(SA)
    assert rows == r
    assert np.all(np.isinf(SAh[:, 1]))
    assert np.all(np.isfinite(np.delete(SAh, 1, axis=1))) and np.all(np.isfinite(host(Sb)))
    x, info = ctx.solve(SA, Sb)
    _reported(host(x), P.info_dict(info))


def test_batched_solve_isolates_the_bad_problem(ctx, orc):
    import torch

    import paper_0812_4547_gb300 as P

    data = [_good(200 + 50 * i, 6 + 3 * i, 10 + i) for i in range(3)]
    bad = data[1][0].copy()
    bad[3, 2] = np.nan
    probs = []
    for i, (S, s) in enumerate(data):
        SA = dev_colmajor(bad if i == 1 else S)
        probs.append((SA, dev_vec(s), torch.empty(S.shape[1], dtype=torch.float64, device="cuda"),
                      torch.zeros(P.INFO_BYTES, dtype=torch.uint8, device="cuda")))
    ctx.solve_batched(probs)
    for i, (S, s) in enumerate(data):
        x, info = host(probs[i][2]), P.info_dict(probs[i][3])
        if i == 1:
            _reported(x, info)
        else:
            _matches_oracle(orc, x, info, S, s)


def test_multi_target_isolates_the_bad_target(ctx, orc):
    import paper_0812_4547_gb300 as P

    rng = np.random.default_rng(4)
    m, d, nrhs = 500, 10, 4
    S = rng.standard_normal((m, d)).astype(np.float32)
    SB = (S.astype(np.float64) @ np.maximum(rng.standard_normal((d, nrhs)), 0)
          + 0.1 * rng.standard_normal((m, nrhs))).astype(np.float32)
    SB[77, 2] = np.inf
    X, raw = ctx.solve_multi(dev_colmajor(S), dev_colmajor(SB))
    X = host(X)
    for t in range(nrhs):
        info = P.info_dict(raw[t])
        if t == 2:
            _reported(X[:, t], info)
        else:
            _matches_oracle(orc, X[:, t], info, S, SB[:, t])


def test_boosted_with_every_run_failing_keeps_run_zero(ctx):
    """No run ends with status OK: the kept run is run 0, reported as such."""
    import paper_0812_4547_gb300 as P

    rng = np.random.default_rng(5)
    n, d = 30000, 5
    A = rng.random((n, d)).astype(np.float32)
    A[999, 3] = np.nan
    b = rng.random(n).astype(np.float32)
    x, resid, best, info = ctx.solve_boosted(dev_colmajor(A), dev_vec(b), 100, 3, seed=6)
    assert int(host(best)[0]) == 0
    _reported(host(x), P.info_dict(info))
    assert not np.any(np.isfinite(host(resid)))


def test_repeated_column_reaches_the_oracle_objective(ctx, orc):
    import paper_0812_4547_gb300 as P

    rng = np.random.default_rng(6)
    S = (rng.random((400, 6)) + 0.05).astype(np.float32)
    S = np.hstack([S, S[:, 2:3]])  # column 6 repeats column 2 (the same FP32 bytes)
    s = (S[:, :6].astype(np.float64) @ np.array([0.3, 0.0, 1.2, 0.5, 0.0, 0.8])
         + 0.05 * rng.standard_normal(400)).astype(np.float32)
    x, info = ctx.solve(dev_colmajor(S), dev_vec(s))
    x, info = host(x), P.info_dict(info)
    xo, io = orc.nnls(S.astype(np.float64), s.astype(np.float64))
    assert info["status"] == io["status"] == 0
    assert np.all(x >= 0) and not (x[2] > 0 and x[6] > 0)
    S64 = S.astype(np.float64)
    # the fitted values S x are unique even though x is not
    assert np.linalg.norm(S64 @ x - S64 @ xo) <= TOL_X * np.linalg.norm(S64 @ xo)
    fo = np.linalg.norm(S64 @ xo - s) ** 2
    assert abs(np.linalg.norm(S64 @ x - s) ** 2 - fo) <= 1e-6 * fo


def test_empty_batches_enqueue_nothing(ctx):
    ctx.sketch_batched([])
    ctx.solve_batched([])
