"""Edge cases of the GPU path against the oracle: the FP64 sketch in
Bernoulli mode (including r >= n, where every row is kept), row counts just
past the small-n limit and just past a power of two (the chunked kernel with
mostly empty chunk groups), an underdetermined sketch (r < d, where the
fitted values and the minimum are unique but x need not be), and host
refusals of empty or oversized problems.
"""
import numpy as np
import pytest

import workloads
from tests.gpu_util import dev_colmajor, dev_vec, host, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_0812_4547_gb300 as P

    c = P.Context(0)
    yield c
    c.close()


def _compare(ctx, orc, A, b, r, seed, mode, tol):
    import paper_0812_4547_gb300 as P

    SA, Sb, idx, rows = ctx.sketch(dev_colmajor(A), dev_vec(b), r, seed, 1,
                                   P.RNNLS_SAMPLE_BERNOULLI if mode else P.RNNLS_SAMPLE_IID)
    SA_o, Sb_o, idx_o = orc.sketch(A, b, r, seed, 1, mode)
    assert rows == len(idx_o) and np.array_equal(host(idx)[:rows], idx_o)
    assert rel_fro(host(SA)[:rows], SA_o) <= tol and rel_fro(host(Sb)[:rows], Sb_o) <= tol
    return rows


@pytest.mark.parametrize("n,d,r", [(4096, 20, 512), (20000, 3, 300), (1000, 4, 2000)])
def test_fp64_sketch_bernoulli(ctx, orc, n, d, r):
    p = workloads.problem(1, n=n, d=d, r=r)
    rows = _compare(ctx, orc, p.A, p.b, r, seed=2, mode=1, tol=1e-12)
    if r >= workloads.next_pow2(n):
        assert rows == workloads.next_pow2(n)


@pytest.mark.parametrize("n", [8193, 12289, 16385, 32769])
@pytest.mark.parametrize("mode", [0, 1])
def test_sizes_just_past_a_boundary(ctx, orc, n, mode):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, 3)).astype(np.float32)
    b = rng.standard_normal(n).astype(np.float32)
    _compare(ctx, orc, A, b, 100, seed=5, mode=mode, tol=1e-5)


def test_underdetermined_sketch(ctx, orc):
    import paper_0812_4547_gb300 as P

    rng = np.random.default_rng(7)
    S = rng.standard_normal((10, 20)).astype(np.float32)
    s = rng.standard_normal(10).astype(np.float32)
    x, info = ctx.solve(dev_colmajor(S), dev_vec(s))
    x, info = host(x), P.info_dict(info)
    xo, io = orc.nnls(S.astype(np.float64), s.astype(np.float64))
    assert info["status"] == io["status"] == 0
    assert np.all(x >= 0)
    S64, s64 = S.astype(np.float64), s.astype(np.float64)
    # the fitted values S x of the minimiser are unique (the objective is
    # strictly convex in S x), and so is the minimum
    assert np.linalg.norm(S64 @ x - S64 @ xo) <= 1e-6 * np.linalg.norm(S64 @ xo)
    fo = np.linalg.norm(S64 @ xo - s64) ** 2
    assert abs(np.linalg.norm(S64 @ x - s64) ** 2 - fo) <= 1e-6 * fo


def test_empty_and_oversized_problems_are_refused(ctx):
    import torch

    import paper_0812_4547_gb300 as P
    from paper_0812_4547_gb300 import _binding as B

    A = torch.zeros((2, 100), device="cuda").t()
    b = torch.zeros(100, device="cuda")
    SA = torch.zeros((2, 10), device="cuda").t()
    Sb = torch.zeros(10, device="cuda")
    x = torch.zeros(2, dtype=torch.float64, device="cuda")
    cases = [
        (B.rnnls_sketch, (ctx.handle, A.data_ptr(), 100, b.data_ptr(), 0, 2, 10, 0, 0, 0, SA.data_ptr(), 10,
                          Sb.data_ptr(), 0, 10), P._binding.RNNLS_EINVAL),  # n_raw = 0
        (B.rnnls_sketch, (ctx.handle, A.data_ptr(), 100, b.data_ptr(), 100, (1 << 20) + 1, 10, 0, 0, 0,
                          SA.data_ptr(), 10, Sb.data_ptr(), 0, 10), P._binding.RNNLS_EUNSUPPORTED),  # d > 2^20
        (B.rnnls_solve, (ctx.handle, SA.data_ptr(), 10, Sb.data_ptr(), 0, 2, x.data_ptr(), 0),
         P._binding.RNNLS_EINVAL),  # r = 0
        (B.rnnls_solve, (ctx.handle, SA.data_ptr(), 10, Sb.data_ptr(), 10, 1025, x.data_ptr(), 0),
         P._binding.RNNLS_EUNSUPPORTED),  # d > 1024
    ]
    for fn, args, status in cases:
        with pytest.raises(P.RNNLSError) as e:
            fn(*args)
        assert e.value.status == status
