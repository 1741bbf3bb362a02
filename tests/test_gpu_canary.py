"""Canary-padded outputs: every call writes inside the output extents its
arguments declare and nowhere else.

Each output buffer is allocated larger than the call is told (a leading
dimension above the row count, trailing elements past a vector's length),
filled with a sentinel, and checked after the call: the declared part holds
the result (checked against the oracle where it is cheap), the padding still
holds the sentinel.  Together with the parity tests (which read only the
declared part) this catches stray writes past an output's end.
"""
import numpy as np
import pytest

from tests.gpu_util import dev_colmajor, dev_vec, host, rel_fro

pytestmark = pytest.mark.gpu

PAD = 5


@pytest.fixture(scope="module")
def ctx():
    import paper_0812_4547_gb300 as P

    c = P.Context(0)
    yield c
    c.close()


def _padded_matrix(rows, cols, dtype=None):
    """(rows, cols) column-major view of a NaN-filled buffer with rows + PAD rows per column."""
    import torch

    buf = torch.full((cols, rows + PAD), float("nan"), dtype=dtype or torch.float32, device="cuda")
    return buf, buf.t()[:rows]


def _padded_vector(n, fill=float("nan"), dtype=None):
    import torch

    buf = torch.full((n + PAD,), fill, dtype=dtype or torch.float32, device="cuda")
    return buf, buf[:n]


def _pad_is_untouched(buf, n, fill=None):
    tail = host(buf)[..., n:]
    return bool(np.all(np.isnan(tail))) if fill is None else bool(np.all(tail == fill))


def _problem(n, d, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, d)).astype(np.float32), rng.standard_normal(n).astype(np.float32)


@pytest.mark.parametrize("n", [3000, 20000])  # the small-n kernel and the chunked kernel
def test_sketch_and_solve_write_only_their_extents(ctx, orc, n):
    import torch

    import paper_0812_4547_gb300 as P

    d, r = 3, 300
    A, b = _problem(n, d, n)
    SA_buf, SA = _padded_matrix(r, d)
    Sb_buf, Sb = _padded_vector(r)
    idx_buf, idx = _padded_vector(r, -7, torch.int32)
    ctx.sketch(dev_colmajor(A), dev_vec(b), r, seed=1, instance=2, SA=SA, Sb=Sb, idx=idx)
    SA_o, Sb_o, idx_o = orc.sketch(A, b, r, 1, 2)
    assert np.array_equal(host(idx), idx_o) and rel_fro(host(SA), SA_o) <= 1e-5 and rel_fro(host(Sb), Sb_o) <= 1e-5
    assert _pad_is_untouched(SA_buf, r) and _pad_is_untouched(Sb_buf, r) and _pad_is_untouched(idx_buf, r, -7)

    x_buf, x = _padded_vector(d, dtype=torch.float64)
    info_buf, info = _padded_vector(P.INFO_BYTES, 0xAB, torch.uint8)
    ctx.solve(SA, Sb, x=x, info=info)
    assert P.info_dict(info)["status"] == 0
    assert _pad_is_untouched(x_buf, d) and _pad_is_untouched(info_buf, P.INFO_BYTES, 0xAB)


def test_bernoulli_sketch_stays_within_its_capacity(ctx):
    import paper_0812_4547_gb300 as P

    n, d, r = 20000, 2, 300
    A, b = _problem(n, d, 5)
    cap = P.bernoulli_capacity(r, P.padded_n(n))
    SA_buf, SA = _padded_matrix(cap, d)
    Sb_buf, Sb = _padded_vector(cap)
    _, _, _, rows = ctx.sketch(dev_colmajor(A), dev_vec(b), r, seed=3, mode=P.RNNLS_SAMPLE_BERNOULLI, SA=SA, Sb=Sb,
                               cap=cap)
    assert 0 < rows <= cap
    assert np.all(np.isfinite(host(SA)[:rows])) and _pad_is_untouched(SA_buf, cap) and _pad_is_untouched(Sb_buf, cap)


def test_multi_target_outputs_stay_within_their_leading_dimensions(ctx):
    import torch

    n, d, nrhs, r = 20000, 4, 3, 256
    rng = np.random.default_rng(6)
    A = rng.random((n, d)).astype(np.float32)
    B = rng.random((n, nrhs)).astype(np.float32)
    SA_buf, SA = _padded_matrix(r, d)
    SB_buf, SB = _padded_matrix(r, nrhs)
    ctx.sketch_multi(dev_colmajor(A), dev_colmajor(B), r, seed=4, SA=SA, SB=SB)
    assert np.all(np.isfinite(host(SA))) and np.all(np.isfinite(host(SB)))
    assert _pad_is_untouched(SA_buf, r) and _pad_is_untouched(SB_buf, r)
    X_buf, X = _padded_matrix(d, nrhs, torch.float64)
    ctx.solve_multi(SA, SB, X=X)
    assert np.all(np.isfinite(host(X))) and _pad_is_untouched(X_buf, d)


def test_batched_and_boosted_outputs_stay_within_their_extents(ctx):
    import torch

    jobs, bufs = [], []
    for i, (n, d, r) in enumerate([(20000, 3, 200), (3000, 2, 100), (70000, 5, 1000)]):
        A, b = _problem(n, d, 10 + i)
        SA_buf, SA = _padded_matrix(r, d)
        Sb_buf, Sb = _padded_vector(r)
        idx_buf, idx = _padded_vector(r, -7, torch.int32)
        jobs.append((dev_colmajor(A), dev_vec(b), r, 7, i, SA, Sb, idx))
        bufs.append((r, SA_buf, Sb_buf, idx_buf))
    ctx.sketch_batched(jobs)
    for r, SA_buf, Sb_buf, idx_buf in bufs:
        assert _pad_is_untouched(SA_buf, r) and _pad_is_untouched(Sb_buf, r) and _pad_is_untouched(idx_buf, r, -7)

    n, d, k = 30000, 4, 3
    A, b = _problem(n, d, 20)
    A = np.abs(A)
    x_buf, x = _padded_vector(d, dtype=torch.float64)
    res_buf, res = _padded_vector(k, dtype=torch.float64)
    best_buf, best = _padded_vector(1, -7, torch.int32)
    ctx.solve_boosted(dev_colmajor(A), dev_vec(b), 200, k, seed=8, x=x, resid=res, best=best)
    assert 0 <= int(host(best)[0]) < k and np.all(np.isfinite(host(res)))
    assert _pad_is_untouched(x_buf, d) and _pad_is_untouched(res_buf, k) and _pad_is_untouched(best_buf, 1, -7)
