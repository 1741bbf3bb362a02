"""The sketch moments of Sec. 3.4 (Q = [SA | Sb]'[SA | Sb], the column
1-norms of SA) formed on the tensor cores (rnnls_gram) against the FP64
oracle's Gram of the same FP32 bytes.

The bound checked is the one the split guarantees: per row at most about
2^-40 max|x_i| max|x_j| from the dropped slices, plus the float-float
rounding of the drained sums (about 2^-44 of sqrt(Q_ii Q_jj))."""
import numpy as np
import pytest

from tests.gpu_util import dev_colmajor, dev_vec, host

pytestmark = pytest.mark.gpu


def _bound(X, Qref):
    m = X.shape[0]
    M = np.abs(X).max(axis=0)
    diag = np.sqrt(np.abs(np.diag(Qref)))
    return 2.0 ** -38 * m * np.outer(M, M) + 1e-12 * np.outer(diag, diag) + 1e-300


def _gram(ctx, SA, Sb):
    Q, colabs = ctx.gram(SA, Sb)
    return host(Q), host(colabs)


def _check(orc, ctx, S32, s32, SA=None, Sb=None):
    SA = dev_colmajor(S32) if SA is None else SA
    Sb = dev_vec(s32) if Sb is None else Sb
    Q, colabs = _gram(ctx, SA, Sb)
    Qr, qr, ssr = orc.gram(S32, s32)
    d = S32.shape[1]
    Qfull = np.zeros((d + 1, d + 1))
    Qfull[:d, :d] = Qr
    Qfull[:d, d] = Qfull[d, :d] = qr
    Qfull[d, d] = ssr
    X = np.column_stack([S32, s32]).astype(np.float64)
    err = np.abs(Q - Qfull)
    bound = _bound(X, Qfull)
    assert np.all(err <= bound), float(np.max(err / bound))
    assert np.array_equal(Q, Q.T)
    want_abs = np.abs(S32.astype(np.float64)).sum(axis=0)
    assert np.allclose(colabs, want_abs, rtol=1e-12, atol=0)
    return Q, Qfull


@pytest.mark.parametrize("r,d", [(1, 1), (7, 3), (32, 16), (33, 17), (1000, 63), (1000, 64), (1000, 65),
                                 (4097, 127), (4097, 128), (4097, 129), (3000, 191), (3000, 192), (2500, 200),
                                 (777, 300), (40000, 40), (100003, 9)])
def test_gram_matches_oracle(orc, r, d):
    import paper_0812_4547_gb300 as P

    rng = np.random.default_rng(r * 1000 + d)
    S32 = (rng.standard_normal((r, d)) * np.exp(rng.standard_normal(d))).astype(np.float32)
    s32 = rng.standard_normal(r).astype(np.float32)
    ctx = P.Context(0)
    try:
        _, Qfull = _check(orc, ctx, S32, s32)
    finally:
        ctx.close()
    # the relative accuracy the Lawson-Hanson parity needs, on Gaussian-like data
    diag = np.sqrt(np.diag(Qfull))
    assert np.max(np.abs(Qfull) / np.outer(diag, diag)) <= 1.0 + 1e-12


def test_gram_of_a_real_sketch(orc):
    """The sketch of a term-document problem (the data the solve sees)."""
    import paper_0812_4547_gb300 as P
    import workloads

    p = workloads.problem(2, n=1 << 15, d=64, r=4096, seed=11)
    A32, b32 = p.A.astype(np.float32), p.b.astype(np.float32)
    SA, Sb, _ = orc.sketch(A32, b32, 4096, seed=3)
    ctx = P.Context(0)
    try:
        Q, Qfull = _check(orc, ctx, SA.astype(np.float32), Sb.astype(np.float32))
        diag = np.sqrt(np.diag(Qfull))
        assert np.max(np.abs(Q - Qfull) / np.outer(diag, diag)) <= 1e-12
    finally:
        ctx.close()


def test_gram_layouts_and_ragged_rows(orc):
    """A leading dimension that is not a multiple of four and an SA that
    starts one float past an aligned address (the unvectorised loads)."""
    import torch

    import paper_0812_4547_gb300 as P

    rng = np.random.default_rng(5)
    r, d, ld = 1037, 70, 1043
    S32 = rng.standard_normal((r, d)).astype(np.float32)
    s32 = rng.standard_normal(r).astype(np.float32)
    buf = torch.zeros((d * ld + 1,), dtype=torch.float32, device="cuda")
    view = buf[1:].view(d, ld).t()[:r]
    view.copy_(torch.from_numpy(S32).cuda())
    ctx = P.Context(0)
    try:
        _check(orc, ctx, S32, s32, SA=view)
    finally:
        ctx.close()


def test_gram_special_columns(orc):
    """A zero column, columns scaled 1e-8 and 1e8, a constant column and
    integer data whose Gram is exact."""
    import paper_0812_4547_gb300 as P

    rng = np.random.default_rng(9)
    r = 2000
    S = rng.standard_normal((r, 6))
    S[:, 0] = 0.0
    S[:, 1] *= 1e-8
    S[:, 2] *= 1e8
    S[:, 3] = 3.0
    S[:, 4] = rng.integers(-1000, 1000, r)
    S32 = S.astype(np.float32)
    s32 = rng.integers(-50, 50, r).astype(np.float32)
    ctx = P.Context(0)
    try:
        Q, Qfull = _check(orc, ctx, S32, s32)
        assert np.all(Q[0, :] == 0.0) and np.all(Q[:, 0] == 0.0)
        # integer columns: every product and sum is an exact integer below 2^53
        for i in (3, 4, 6):
            for j in (3, 4, 6):
                assert Q[i, j] == Qfull[i, j]
    finally:
        ctx.close()


def test_gram_non_finite_column():
    """A NaN or an infinity in a column makes that column's entries of Q NaN
    (the solve then reports ENONFINITE)."""
    import paper_0812_4547_gb300 as P

    rng = np.random.default_rng(2)
    for bad in (np.nan, np.inf):
        S32 = rng.standard_normal((500, 5)).astype(np.float32)
        S32[123, 2] = bad
        ctx = P.Context(0)
        try:
            Q, _ = _gram(ctx, dev_colmajor(S32), dev_vec(rng.standard_normal(500).astype(np.float32)))
        finally:
            ctx.close()
        assert np.all(np.isnan(Q[2, :])) and np.all(np.isnan(Q[:, 2]))
        assert np.all(np.isfinite(np.delete(np.delete(Q, 2, 0), 2, 1)))


def test_gram_repeated_calls_and_argument_errors():
    import paper_0812_4547_gb300 as P
    from paper_0812_4547_gb300 import _binding as B

    rng = np.random.default_rng(4)
    S32 = rng.standard_normal((5000, 33)).astype(np.float32)
    s32 = rng.standard_normal(5000).astype(np.float32)
    SA, Sb = dev_colmajor(S32), dev_vec(s32)
    ctx = P.Context(0)
    try:
        Q0, _ = _gram(ctx, SA, Sb)
        for _ in range(3):
            Q1, _ = _gram(ctx, SA, Sb)
            assert np.array_equal(Q0, Q1)  # deterministic: fixed slicing and summation order
        lib = B.lib()
        import ctypes

        assert lib.rnnls_gram(ctypes.c_void_p(ctx.handle), ctypes.c_void_p(SA.data_ptr()), 5000,
                              ctypes.c_void_p(Sb.data_ptr()), 5000, 0, ctypes.c_void_p(1), None) == B.RNNLS_EINVAL
        assert lib.rnnls_gram(ctypes.c_void_p(ctx.handle), ctypes.c_void_p(SA.data_ptr()), 4999,
                              ctypes.c_void_p(Sb.data_ptr()), 5000, 33, ctypes.c_void_p(1), None) == B.RNNLS_EINVAL
        assert lib.rnnls_gram(ctypes.c_void_p(ctx.handle), ctypes.c_void_p(SA.data_ptr()), 5000,
                              ctypes.c_void_p(Sb.data_ptr()), 5000, 1025, ctypes.c_void_p(1),
                              None) == B.RNNLS_EUNSUPPORTED
    finally:
        ctx.close()
