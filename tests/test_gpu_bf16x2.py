"""RNNLS_PREC_BF16X2: the split-precision form of the sketch (Sec. 3.4's
preconditioning step with the first 64-point factor of each 4096-row chunk's
Walsh-Hadamard transform on the tensor cores: values split into hi + lo BF16
pairs, multiplied by H_64, whose +-1 entries BF16 holds exactly, with FP32
accumulation).

Against the FP64 oracle's sketch of the same FP32 bytes: rows bit-exact
(the mode changes no sampling), SA and Sb within 5e-4 relative Frobenius
(the bound the split-precision form is held to), and within 2e-5 as well,
the split's own scale (2^-18 per value plus FP32 accumulation), so that a
lost lo half (error near 2^-9) would fail.  Every case also checks that the
result differs from the FP32 mode's: the tensor-core pass ran."""
import math

import numpy as np
import pytest

import workloads
from tests.gpu_util import dev_colmajor, dev_vec, host, rel_fro

pytestmark = pytest.mark.gpu

TOL_SPLIT = 5e-4
TOL_SCALE = 2e-5


@pytest.fixture(scope="module")
def ctx():
    import paper_0812_4547_gb300 as P

    c = P.Context(0)
    yield c
    c.close()


def both_modes(ctx, A, b, r, seed, inst, mode=0):
    import paper_0812_4547_gb300 as P

    smode = P.RNNLS_SAMPLE_BERNOULLI if mode else P.RNNLS_SAMPLE_IID
    Ad, bd = dev_colmajor(A), dev_vec(b)
    SA, Sb, idx, rows = ctx.sketch(Ad, bd, r, seed, inst, smode, prec=P.RNNLS_PREC_BF16X2)
    SA32, Sb32, idx32, rows32 = ctx.sketch(Ad, bd, r, seed, inst, smode)
    assert rows == rows32
    return host(SA)[:rows], host(Sb)[:rows], host(idx)[:rows], host(SA32)[:rows], host(idx32)[:rows]


CASES = [
    (16384, 1, 1),            # one step, one row
    (16384, 5, 300),          # one step per column
    (50001, 7, 1000),         # ragged tail, several steps
    ((1 << 16) + 3, 3, 9000),  # 40 rows per thread in registers
    (1 << 15, 4, 16384),      # rows in TMEM, full-step mode
    (70000, 3, 30000),        # two plan groups (more rows than the mode's TMEM share)
    (300000, 2, 2500),        # columns split over many blocks (partial sums)
]


@pytest.mark.parametrize("n,d,r", CASES)
def test_split_precision_sketch_matches_oracle(ctx, orc, n, d, r):
    rng = np.random.default_rng(n + 3 * d + r)
    A = rng.standard_normal((n, d)).astype(np.float32)
    b = rng.standard_normal(n).astype(np.float32)
    SA, Sb, idx, SA32, idx32 = both_modes(ctx, A, b, r, seed=21, inst=3)
    SA_o, Sb_o, idx_o = orc.sketch(A, b, r, 21, 3, 0)
    assert np.array_equal(idx, idx_o) and np.array_equal(idx32, idx_o)
    e_sa, e_sb = rel_fro(SA, SA_o), rel_fro(Sb, Sb_o)
    assert e_sa <= TOL_SPLIT and e_sb <= TOL_SPLIT
    assert e_sa <= TOL_SCALE and e_sb <= TOL_SCALE, (e_sa, e_sb)
    if SA.size >= 256:  # a handful of values may round the same in both modes
        assert not np.array_equal(SA, SA32)  # the tensor-core pass ran


def test_split_precision_bernoulli_rows(ctx, orc):
    rng = np.random.default_rng(8)
    n, d, r = (1 << 15) + 9, 4, 2000
    A = rng.standard_normal((n, d)).astype(np.float32)
    b = rng.standard_normal(n).astype(np.float32)
    SA, Sb, idx, SA32, _ = both_modes(ctx, A, b, r, seed=4, inst=0, mode=1)
    SA_o, Sb_o, idx_o = orc.sketch(A, b, r, 4, 0, 1)
    assert np.array_equal(idx, idx_o)
    assert rel_fro(SA, SA_o) <= TOL_SCALE and rel_fro(Sb, Sb_o) <= TOL_SCALE
    assert not np.array_equal(SA, SA32)


def test_split_precision_unaligned_input(ctx, orc):
    """A and b not 16-byte aligned: the chunks are loaded with plain loads,
    then the same tensor-core pass."""
    import torch

    import paper_0812_4547_gb300 as P

    rng = np.random.default_rng(9)
    n, d, r = 40000, 3, 700
    A = rng.standard_normal((n, d)).astype(np.float32)
    b = rng.standard_normal(n).astype(np.float32)
    buf = torch.zeros(d * (n + 1) + 1, device="cuda")
    Av = torch.as_strided(buf[1:], (n, d), (1, n + 1))
    Av.copy_(torch.from_numpy(A).cuda())
    bbuf = torch.zeros(n + 1, device="cuda")
    bv = bbuf[1:]
    bv.copy_(torch.from_numpy(b).cuda())
    SA, Sb, idx, _ = ctx.sketch(Av, bv, r, 6, 1, prec=P.RNNLS_PREC_BF16X2)
    SA_o, Sb_o, idx_o = orc.sketch(A, b, r, 6, 1, 0)
    assert np.array_equal(host(idx), idx_o)
    assert rel_fro(host(SA), SA_o) <= TOL_SCALE and rel_fro(host(Sb), Sb_o) <= TOL_SCALE


def test_split_precision_small_n_is_fp32(ctx, orc):
    """Padded n <= 8192 (whole column in shared memory): the flag is
    accepted and the FP32 transform runs."""
    rng = np.random.default_rng(10)
    A = rng.standard_normal((5000, 3)).astype(np.float32)
    b = rng.standard_normal(5000).astype(np.float32)
    SA, Sb, idx, SA32, _ = both_modes(ctx, A, b, 300, seed=2, inst=0)
    assert np.array_equal(SA, SA32)
    SA_o, _, _ = orc.sketch(A, b, 300, 2, 0, 0)
    assert rel_fro(SA, SA_o) <= 1e-5


def test_split_precision_flag_refusals(ctx):
    import torch

    import paper_0812_4547_gb300 as P
    from paper_0812_4547_gb300 import _binding as B

    A = torch.zeros((4, 100), device="cuda").t()
    b = torch.zeros(100, device="cuda")
    SA = torch.zeros((4, 10), device="cuda").t()
    Sb = torch.zeros(10, device="cuda")
    # FP64 data has no split-precision mode; unknown bits are refused
    A64 = torch.zeros((4, 100), dtype=torch.float64, device="cuda").t()
    b64 = torch.zeros(100, dtype=torch.float64, device="cuda")
    SA64 = torch.zeros((4, 10), dtype=torch.float64, device="cuda").t()
    Sb64 = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(P.RNNLSError) as e:
        B.rnnls_sketch_f64(ctx.handle, A64.data_ptr(), 100, b64.data_ptr(), 100, 4, 10, 0, 0, B.RNNLS_PREC_BF16X2,
                           SA64.data_ptr(), 10, Sb64.data_ptr(), 0, 10)
    assert e.value.status == B.RNNLS_EINVAL
    with pytest.raises(P.RNNLSError) as e:
        B.rnnls_sketch(ctx.handle, A.data_ptr(), 100, b.data_ptr(), 100, 4, 10, 0, 0, 4, SA.data_ptr(), 10,
                       Sb.data_ptr(), 0, 10)
    assert e.value.status == B.RNNLS_EINVAL
    job = B.rnnls_sketch_job(A.data_ptr(), 100, b.data_ptr(), 100, 4, 10, 0, 0, SA.data_ptr(), 10, Sb.data_ptr(),
                             torch.zeros(10, dtype=torch.int32, device="cuda").data_ptr())
    with pytest.raises(P.RNNLSError) as e:
        B.rnnls_sketch_batched(ctx.handle, [job], 1)
    assert e.value.status == B.RNNLS_EINVAL


def test_split_precision_batched_matches_single(ctx, orc):
    """rnnls_sketch_batched_ex in the split-precision mode: each instance as
    the one-instance call in the same mode gives it (rows bit-exact, values
    to FP32 summation order), and the oracle's sketch within the mode's
    bound; uneven sizes including two plan groups and a small-n instance."""
    import torch

    import paper_0812_4547_gb300 as P

    rng = np.random.default_rng(12)
    shapes = [(40000, 30, 8192), (20000, 12, 30000), (70000, 9, 4096), (6000, 5, 500), (1 << 17, 3, 16384)]
    inst = []
    for n, d, r in shapes:
        A = rng.standard_normal((n, d)).astype(np.float32)
        b = rng.standard_normal(n).astype(np.float32)
        inst.append((A, b, r, dev_colmajor(A), dev_vec(b)))
    items = []
    for i, (A, b, r, Ad, bd) in enumerate(inst):
        d = A.shape[1]
        items.append((Ad, bd, r, 5, i, torch.empty((d, r), device="cuda").t(), torch.empty(r, device="cuda"),
                      torch.empty(r, dtype=torch.int32, device="cuda")))
    ctx.sketch_batched(items, prec=P.RNNLS_PREC_BF16X2)
    torch.cuda.synchronize()
    for (A, b, r, Ad, bd), (_, _, _, seed, i, SA, Sb, idx) in zip(inst, items):
        SA1, Sb1, idx1, _ = ctx.sketch(Ad, bd, r, seed, i, prec=P.RNNLS_PREC_BF16X2)
        assert np.array_equal(host(idx), host(idx1))
        assert rel_fro(host(SA), host(SA1).astype(np.float64)) <= 1e-6
        SA_o, Sb_o, idx_o = orc.sketch(A, b, r, seed, i, 0)
        assert np.array_equal(host(idx), idx_o)
        assert rel_fro(host(SA), SA_o) <= TOL_SCALE and rel_fro(host(Sb), Sb_o) <= TOL_SCALE


def test_split_precision_workload_three_sampled_entries(ctx, orc):
    """Workload 3 at full size (2^22 x 128, r = 8192) in the benchmark's
    launch configuration; rows bit-exact, sampled entries against the
    definition within the mode's bound."""
    import paper_0812_4547_gb300 as P

    p = workloads.problem(3)
    A = dev_colmajor(p.A)
    b = dev_vec(p.b)
    SA, Sb, idx, _ = ctx.sketch(A, b, p.r, seed=7, instance=0, prec=P.RNNLS_PREC_BF16X2)
    idx_o = orc.sample(7, 0, P.padded_n(p.n), p.r)
    assert np.array_equal(host(idx), idx_o)
    SAh, Sbh = host(SA), host(Sb)
    sc = 1 / math.sqrt(p.r)
    rng = np.random.default_rng(3)
    for _ in range(12):
        k = int(rng.integers(p.r))
        j = int(rng.integers(p.d + 1))
        col = p.A[:, j] if j < p.d else p.b
        want = orc.sketch_entry(col, 7, 0, int(idx_o[k]), sc)
        got = SAh[k, j] if j < p.d else Sbh[k]
        assert abs(got - want) <= TOL_SCALE * sc * np.linalg.norm(col.astype(np.float64))


def test_split_precision_workload_five_sampled_entries(orc):
    """Instances of workload 5's recipe at their real sizes (the benchmark's
    device generator, one batched launch in the split-precision mode): the
    largest-r instances (two plan groups in this mode) and a spread of the
    others; rows bit-exact, sampled entries against the definition."""
    import torch

    import bench
    import paper_0812_4547_gb300 as P

    shapes = workloads.batch_shapes()
    big_r = [i for i, s in enumerate(shapes) if s[2] >= 32768][:3]
    pick = sorted(set(big_r) | set(range(0, len(shapes), 64)))
    insts = bench.device_batch(shapes, 5, torch.device("cuda"), only=pick)
    c = P.Context(0)
    try:
        items = []
        for i, (A, b, r) in zip(pick, insts):
            d = A.shape[1]
            items.append((A, b, r, 5, i, torch.empty((d, r), device="cuda").t(), torch.empty(r, device="cuda"),
                          torch.empty(r, dtype=torch.int32, device="cuda")))
        c.sketch_batched(items, prec=P.RNNLS_PREC_BF16X2)
        torch.cuda.synchronize()
    finally:
        c.close()
    rng = np.random.default_rng(17)
    for (A, b, r, seed, inst, SA, Sb, idx) in items:
        n_raw, d = A.shape
        idx_o = orc.sample(seed, inst, P.padded_n(n_raw), r)
        assert np.array_equal(host(idx), idx_o)
        sc = 1 / math.sqrt(r)
        for _ in range(2):
            k = int(rng.integers(r))
            j = int(rng.integers(d + 1))
            col = host(A[:, j] if j < d else b).astype(np.float64)
            want = orc.sketch_entry(col, seed, inst, int(idx_o[k]), sc)
            got = host(SA)[k, j] if j < d else host(Sb)[k]
            assert abs(got - want) <= TOL_SCALE * sc * np.linalg.norm(col)
