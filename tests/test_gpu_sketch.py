"""GPU parity of the sketch (Alg. 1 steps 1-4) against the FP64 oracle.

Sampled rows must match bit-exactly; SA and Sb within 1e-5 relative
Frobenius error for the FP32 path (the oracle reads the same FP32 bytes,
promoted exactly to FP64) and 1e-12 for the FP64 path.
"""
import math

import numpy as np
import pytest

import workloads
from tests.gpu_util import dev_colmajor, dev_vec, host, rel_fro

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
TOL_F64 = 1e-12


@pytest.fixture(scope="module")
def ctx():
    import paper_0812_4547_gb300 as P

    c = P.Context(0)
    yield c
    c.close()


def run_case(ctx, orc, A, b, r, seed, inst, mode, dtype=np.float32, tol=TOL_F32):
    import paper_0812_4547_gb300 as P

    A = np.asarray(A, dtype=dtype)
    b = np.asarray(b, dtype=dtype)
    SA, Sb, idx, rows = ctx.sketch(dev_colmajor(A), dev_vec(b), r, seed, inst,
                                   P.RNNLS_SAMPLE_BERNOULLI if mode else P.RNNLS_SAMPLE_IID)
    SA_o, Sb_o, idx_o = orc.sketch(A, b, r, seed, inst, mode)
    assert rows == len(idx_o)
    assert np.array_equal(host(idx)[:rows], idx_o)
    assert rel_fro(host(SA)[:rows], SA_o) <= tol
    assert rel_fro(host(Sb)[:rows], Sb_o) <= tol
    return host(SA)[:rows], host(Sb)[:rows]


SMALL = [(1, 1, 1), (3, 2, 5), (64, 3, 16), (1000, 4, 100), (4096, 20, 512), (8192, 7, 300), (5000, 2, 8000)]


@pytest.mark.parametrize("n,d,r", SMALL)
@pytest.mark.parametrize("mode", [0, 1])
def test_small_n(ctx, orc, n, d, r, mode):
    rng = np.random.default_rng(n + 7 * d + r)
    run_case(ctx, orc, rng.standard_normal((n, d)), rng.standard_normal(n), r, seed=3, inst=1, mode=mode)


CHUNKED = [
    (16384, 1, 1), (16384, 3, 100), (20000, 5, 777), (65536, 8, 4096), (1 << 18, 4, 6000),
    (300000, 2, 9000), (1 << 17, 3, 21000), (1 << 16, 2, 70000),
]


@pytest.mark.parametrize("n,d,r", CHUNKED)
@pytest.mark.parametrize("mode", [0, 1])
def test_chunked(ctx, orc, n, d, r, mode):
    rng = np.random.default_rng(n + d + r)
    A = rng.standard_normal((n, d))
    b = rng.standard_normal(n)
    run_case(ctx, orc, A, b, r, seed=11, inst=2, mode=mode)


def test_termdoc_workload_scaled(ctx, orc):
    p = workloads.problem(2, n=1 << 16, d=64, r=4096)
    run_case(ctx, orc, p.A, p.b, p.r, seed=0, inst=0, mode=0)


def test_unaligned_and_strided_inputs(ctx, orc):
    import torch

    import paper_0812_4547_gb300 as P

    rng = np.random.default_rng(5)
    n, d, r = 40000, 3, 500
    A = rng.standard_normal((n, d)).astype(np.float32)
    b = rng.standard_normal(n).astype(np.float32)
    # leading dimension n + 3 (not a multiple of 4) and a b that starts 4 bytes in
    big = torch.zeros((d, n + 3), dtype=torch.float32, device="cuda")
    big[:, :n] = torch.from_numpy(A.T).cuda()
    At = big.t()[:n]
    bb = torch.zeros(n + 1, dtype=torch.float32, device="cuda")
    bb[1:] = torch.from_numpy(b).cuda()
    SA, Sb, idx, rows = ctx.sketch(At, bb[1:], r, 4, 0, P.RNNLS_SAMPLE_IID)
    SA_o, Sb_o, idx_o = orc.sketch(A, b, r, 4, 0, 0)
    assert np.array_equal(host(idx), idx_o)
    assert rel_fro(host(SA), SA_o) <= TOL_F32
    assert rel_fro(host(Sb), Sb_o) <= TOL_F32


@pytest.mark.parametrize("n,d,r", [(4096, 20, 512), (100, 3, 50), (20000, 3, 300),
                                   (300000, 4, 5000),   # one pass, four chunk groups per column
                                   (70000, 2, 16384),   # one pass, the largest r it keeps in shared memory
                                   (50000, 3, 20000)])  # larger r: the two-pass path
def test_fp64_path(ctx, orc, n, d, r):
    p = workloads.problem(1, n=n, d=d, r=r)
    run_case(ctx, orc, p.A, p.b, r, seed=0, inst=0, mode=0, dtype=np.float64, tol=TOL_F64)


def test_keep_all_rows(ctx, orc):
    rng = np.random.default_rng(6)
    A = rng.random((3000, 4))
    b = rng.random(3000)
    SA, Sb = run_case(ctx, orc, A, b, 4096, seed=1, inst=0, mode=1)
    assert SA.shape[0] == 4096


def test_deterministic(ctx):
    rng = np.random.default_rng(9)
    A = dev_colmajor(rng.standard_normal((70000, 5)), np.float32)
    b = dev_vec(rng.standard_normal(70000), np.float32)
    s1 = ctx.sketch(A, b, 3000, 5)
    s2 = ctx.sketch(A, b, 3000, 5)
    assert np.array_equal(host(s1[0]), host(s2[0]))
    assert np.array_equal(host(s1[1]), host(s2[1]))


def test_capacity_error(ctx):
    import paper_0812_4547_gb300 as P

    rng = np.random.default_rng(10)
    A = dev_colmajor(rng.standard_normal((1 << 15, 2)), np.float32)
    b = dev_vec(rng.standard_normal(1 << 15), np.float32)
    with pytest.raises(P.RNNLSError) as e:
        ctx.sketch(A, b, 4000, 1, mode=P.RNNLS_SAMPLE_BERNOULLI, cap=3000)
    assert e.value.status == 2


def test_invalid_arguments(ctx):
    import torch

    import paper_0812_4547_gb300 as P
    from paper_0812_4547_gb300 import _binding as B

    A = torch.zeros((4, 100), device="cuda").t()
    b = torch.zeros(100, device="cuda")
    SA = torch.zeros((4, 10), device="cuda").t()
    Sb = torch.zeros(10, device="cuda")
    for bad in [dict(r=0), dict(lda=50), dict(cap=5), dict(d=0), dict(flags=8)]:
        args = dict(lda=100, d=4, r=10, flags=0, cap=10)
        args.update(bad)
        with pytest.raises(P.RNNLSError) as e:
            B.rnnls_sketch(ctx.handle, A.data_ptr(), args["lda"], b.data_ptr(), 100, args["d"], args["r"], 0, 0,
                           args["flags"], SA.data_ptr(), 10, Sb.data_ptr(), 0, args["cap"])
        assert e.value.status == 1
    with pytest.raises(P.RNNLSError):
        B.rnnls_sketch(ctx.handle, 0, 100, b.data_ptr(), 100, 4, 10, 0, 0, 0, SA.data_ptr(), 10, Sb.data_ptr(), 0, 10)


@pytest.mark.parametrize("config", [2, 3])
def test_full_size_sampled_entries(ctx, orc, config):
    # full workload size, launch configuration of the benchmark; entries
    # checked one by one against the definition (O(n) each)
    import paper_0812_4547_gb300 as P

    p = workloads.problem(config)
    A = dev_colmajor(p.A)
    b = dev_vec(p.b)
    SA, Sb, idx, rows = ctx.sketch(A, b, p.r, seed=7, instance=0)
    idx_o = orc.sample(7, 0, P.padded_n(p.n), p.r)
    assert np.array_equal(host(idx), idx_o)
    SAh, Sbh = host(SA), host(Sb)
    sc = 1 / math.sqrt(p.r)
    rng = np.random.default_rng(1)
    for _ in range(12):
        k = int(rng.integers(p.r))
        j = int(rng.integers(p.d + 1))
        col = p.A[:, j] if j < p.d else p.b
        want = orc.sketch_entry(col, 7, 0, int(idx_o[k]), sc)
        got = SAh[k, j] if j < p.d else Sbh[k]
        # an entry is a +-1 sum of n terms: its typical size is sc * ||col||
        assert abs(got - want) <= 1e-5 * sc * np.linalg.norm(col.astype(np.float64))
    # column norms: ||SX e_j||^2 estimates ||X e_j||^2 (Lemma 1) -- sanity bound
    nrm = np.linalg.norm(SAh[:, 0]) / np.linalg.norm(p.A[:, 0].astype(np.float64))
    assert 0.7 < nrm < 1.3


@pytest.mark.parametrize("sms", [1, 3, 17, 150])
def test_sketch_sm_cap(orc, sms):
    """A cap on the sketch's SMs changes how columns are split over blocks
    (whole columns per block when columns outnumber 8 blocks per SM-slot,
    balanced step ranges with partial sums otherwise), not the result."""
    import paper_0812_4547_gb300 as P

    c = P.Context(0)
    try:
        c.set_sketch_sms(sms)
        rng = np.random.default_rng(sms)
        for n, d, r in [((1 << 18) + 5, 6, 3000), (50000, 40, 1500)]:
            run_case(c, orc, rng.standard_normal((n, d)), rng.standard_normal(n), r, seed=sms, inst=4, mode=0)
    finally:
        c.close()


def test_plan_event_is_recorded_and_changes_nothing():
    """rnnls_set_plan_event: the event is recorded by every FP32 sketch call
    (with and without a plan) and the sketch is the one without it."""
    import torch

    import paper_0812_4547_gb300 as P

    c = P.Context(0)
    try:
        rng = np.random.default_rng(3)
        for n, d, r in [((1 << 17) + 9, 5, 700), (3000, 4, 200)]:
            A = dev_colmajor(rng.standard_normal((n, d)), np.float32)
            b = dev_vec(rng.standard_normal(n), np.float32)
            SA0, Sb0, idx0, _ = c.sketch(A, b, r, seed=5, instance=1)
            ev = torch.cuda.Event()
            ev.record(torch.cuda.current_stream())
            torch.cuda.synchronize()
            c.set_plan_event(ev)
            side = torch.cuda.Stream()
            side.wait_event(ev)  # a stream that follows the plan launch
            SA1, Sb1, idx1, _ = c.sketch(A, b, r, seed=5, instance=1)
            side.wait_event(ev)
            c.set_plan_event(None)
            torch.cuda.synchronize()
            assert ev.query()
            assert np.array_equal(host(idx0), host(idx1))
            assert np.array_equal(host(SA0), host(SA1))
            assert np.array_equal(host(Sb0), host(Sb1))
    finally:
        c.close()


def test_largest_supported_n(ctx, orc):
    """n_raw = 2^28, the largest row count the library takes (one column of A
    and b, 1 GiB each): rows bit-exact, sampled entries against the
    definition; one row more is refused before anything runs."""
    import torch

    import paper_0812_4547_gb300 as P
    from paper_0812_4547_gb300 import _binding as B

    n, r = 1 << 28, 2048
    rng = np.random.default_rng(28)
    a_h = rng.random(n, dtype=np.float32)
    b_h = rng.random(n, dtype=np.float32) - 0.5
    A = torch.from_numpy(a_h).cuda().reshape(1, n).t()
    b = torch.from_numpy(b_h).cuda()
    SA, Sb, idx, rows = ctx.sketch(A, b, r, seed=3, instance=2)
    idx_o = orc.sample(3, 2, n, r)
    assert np.array_equal(host(idx), idx_o)
    SAh, Sbh = host(SA), host(Sb)
    sc = 1 / math.sqrt(r)
    for col_h, got_col in ((a_h, SAh[:, 0]), (b_h, Sbh)):
        col = col_h.astype(np.float64)
        tol = 1e-5 * sc * np.linalg.norm(col)
        for k in (0, 977, r - 1):
            want = orc.sketch_entry(col, 3, 2, int(idx_o[k]), sc)
            assert abs(got_col[k] - want) <= tol
        del col
    del A, b, SA, Sb
    torch.cuda.empty_cache()
    small = torch.zeros(16, device="cuda")
    out = torch.zeros(16, device="cuda")
    with pytest.raises(P.RNNLSError) as e:
        B.rnnls_sketch(ctx.handle, small.data_ptr(), n + 1, small.data_ptr(), n + 1, 1, 8, 0, 0, 0, out.data_ptr(), 8,
                       out.data_ptr(), 0, 8)
    assert e.value.status == B.RNNLS_EUNSUPPORTED
