"""GPU parity of the batched sketch (rnnls_sketch_batched) on uneven instances.

Every instance of a batch must get the sketch rnnls_sketch gives it alone:
the same rows bit for bit, SA and Sb within FP32 summation-order noise
(1e-6 relative), and within the oracle tolerance of the FP64 oracle.
"""
import numpy as np
import pytest

from tests.gpu_util import dev_colmajor, dev_vec, host, rel_fro

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
TOL_SAME = 1e-6

# (n_raw, d, r): chunked sizes with few and many rows per thread (TMEM), a
# ragged tail, one below the chunked size, one with a leading dimension not a
# multiple of 4 (plain loads)
SHAPES = [((1 << 14) + 7, 3, 300), (1 << 16, 17, 4096), (70001, 9, 20000), (5000, 4, 700), (1 << 17, 40, 9000),
          (40000, 2, 33000)]
# few steps (188) of very different cost for 152 blocks: the cost-weighted
# block ranges are clamped to one step each and short units are split
FEW = [(20000, 30, 32768), (16385, 40, 2048), (50000, 10, 8192)]


@pytest.fixture(scope="module")
def ctx():
    import paper_0812_4547_gb300 as P

    c = P.Context(0)
    yield c
    c.close()


def _make(rng, n, d, r, pad=0):
    import torch

    A = rng.standard_normal((n, d)).astype(np.float32)
    b = rng.standard_normal(n).astype(np.float32)
    if pad:
        buf = torch.zeros((d, n + pad), dtype=torch.float32, device="cuda")
        buf[:, :n] = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
        A_d = buf.t()[:n]
    else:
        A_d = dev_colmajor(A)
    return A, b, A_d, dev_vec(b)


@pytest.mark.parametrize("shapes", [SHAPES, FEW], ids=["uneven", "few-steps"])
def test_batched_equals_one_by_one(ctx, orc, shapes):
    import torch

    rng = np.random.default_rng(5)
    items, data = [], []
    for t, (n, d, r) in enumerate(shapes):
        A, b, A_d, b_d = _make(rng, n, d, r, pad=3 if t == 2 else 0)
        SA = torch.full((d, r), float("nan"), device="cuda").t()
        Sb = torch.full((r,), float("nan"), device="cuda")
        idx = torch.full((r,), -1, dtype=torch.int32, device="cuda")
        items.append((A_d, b_d, r, 100 + t, t, SA, Sb, idx))
        data.append((A, b, A_d, b_d, r, 100 + t, t))
    for rep in range(2):  # twice: the partial-sum counters must be left at zero
        ctx.sketch_batched(items)
        torch.cuda.synchronize()
        for (A, b, A_d, b_d, r, seed, inst), it in zip(data, items):
            SA1, Sb1, idx1, _ = ctx.sketch(A_d, b_d, r, seed=seed, instance=inst)
            assert np.array_equal(host(it[7]), host(idx1))
            assert rel_fro(host(it[5]), host(SA1).astype(np.float64)) <= TOL_SAME
            assert rel_fro(host(it[6]), host(Sb1).astype(np.float64)) <= TOL_SAME
    for (A, b, A_d, b_d, r, seed, inst), it in list(zip(data, items))[:3]:
        SA_o, Sb_o, idx_o = orc.sketch(A.astype(np.float64), b.astype(np.float64), r, seed, inst)
        assert np.array_equal(host(it[7]), idx_o)
        assert rel_fro(host(it[5]), SA_o) <= TOL_F32
        assert rel_fro(host(it[6]), Sb_o) <= TOL_F32


def test_batched_rejects_bad_job(ctx):
    import torch

    import paper_0812_4547_gb300 as P

    A = torch.zeros((2, 20000), device="cuda").t()
    b = torch.zeros(20000, device="cuda")
    SA = torch.zeros((2, 100), device="cuda").t()
    Sb = torch.zeros(100, device="cuda")
    idx = torch.zeros(100, dtype=torch.int32, device="cuda")
    with pytest.raises(P.RNNLSError):
        ctx.sketch_batched([(A, b, 100, 1, 0, SA, Sb, idx), (A, b, 0, 1, 0, SA, Sb, idx)])


def test_batched_workload_five_shapes_sampled_entries(orc):
    """The first 16 instances of workload 5's recipe at their real sizes
    (the benchmark's device generator and launch): every instance's rows
    bit-exact and two sampled entries against the definition."""
    import math

    import torch

    import bench
    import paper_0812_4547_gb300 as P
    import workloads

    shapes = workloads.batch_shapes(count=16)
    insts = bench.device_batch(shapes, 5, torch.device("cuda"))
    c = P.Context(0)
    try:
        items = []
        for i, (A, b, r) in enumerate(insts):
            d = A.shape[1]
            items.append((A, b, r, 5, i, torch.empty((d, r), device="cuda").t(), torch.empty(r, device="cuda"),
                          torch.empty(r, dtype=torch.int32, device="cuda")))
        c.sketch_batched(items)
        torch.cuda.synchronize()
    finally:
        c.close()
    rng = np.random.default_rng(16)
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
            assert abs(got - want) <= 1e-5 * sc * np.linalg.norm(col)


def test_batched_solve_from_device_descriptors(orc):
    """rnnls_solve_batched_device: the descriptors in device memory, the plan
    made on the device; results equal the host-descriptor call's, and a
    descriptor outside the bounds is refused through its own info."""
    import ctypes

    import torch

    import paper_0812_4547_gb300 as P
    from paper_0812_4547_gb300 import _binding as B

    rng = np.random.default_rng(17)
    shapes = [(4096, 20), (2000, 64), (9000, 130), (300, 7), (16384, 200)]
    probs, outs = [], []
    for r, d in shapes:
        SA = dev_colmajor(rng.standard_normal((r, d)) * np.exp(rng.standard_normal(d)), np.float32)
        Sb = dev_vec(rng.standard_normal(r), np.float32)
        probs.append((SA, Sb, r, d))
        outs.append((torch.empty(d, dtype=torch.float64, device="cuda"), torch.zeros(P.INFO_BYTES, dtype=torch.uint8,
                                                                                     device="cuda"),
                     torch.empty(d, dtype=torch.float64, device="cuda"), torch.zeros(P.INFO_BYTES, dtype=torch.uint8,
                                                                                     device="cuda")))
    ctx = P.Context(0)
    try:
        ctx.solve_batched([(SA, Sb, o[0], o[1]) for (SA, Sb, r, d), o in zip(probs, outs)])
        descs = [B.rnnls_problem(SA.data_ptr(), SA.stride(1), Sb.data_ptr(), r, d, o[2].data_ptr(), o[3].data_ptr())
                 for (SA, Sb, r, d), o in zip(probs, outs)]
        # one more descriptor whose d exceeds the bound: refused, the others solved
        bad_x = torch.full((300,), 7.0, dtype=torch.float64, device="cuda")
        bad_info = torch.zeros(P.INFO_BYTES, dtype=torch.uint8, device="cuda")
        SA0, Sb0 = probs[0][0], probs[0][1]
        descs.append(B.rnnls_problem(SA0.data_ptr(), SA0.stride(1), Sb0.data_ptr(), 4096, 300, bad_x.data_ptr(),
                                     bad_info.data_ptr()))
        arr = (B.rnnls_problem * len(descs))(*descs)
        d_arr = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).cuda()
        B.rnnls_solve_batched_device(ctx.handle, d_arr.data_ptr(), len(descs), 16384, 200)
        torch.cuda.synchronize()
        for (SA, Sb, r, d), o in zip(probs, outs):
            x_host, x_dev = host(o[0]), host(o[2])
            assert np.array_equal(x_host, x_dev)
            assert P.info_dict(o[3])["status"] == 0
        assert P.info_dict(bad_info)["status"] == B.RNNLS_EINVAL
        assert np.all(host(bad_x) == 7.0)
        assert B.lib().rnnls_solve_batched_device(ctypes.c_void_p(ctx.handle), ctypes.c_void_p(d_arr.data_ptr()), 2,
                                                  100, 1025, 0) == B.RNNLS_EUNSUPPORTED
        assert B.lib().rnnls_solve_batched_device(ctypes.c_void_p(ctx.handle), None, 2, 100, 10, 0) == B.RNNLS_EINVAL
    finally:
        ctx.close()
