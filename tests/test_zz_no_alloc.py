"""rnnls_sketch_noalloc: the sketch entry point for callers that cannot
allocate device memory at call time (frozen or fully reserved memory pools,
allocation-free real-time loops).  It must give the same sketch as
rnnls_sketch and as the FP64 oracle, call after call, while its scratch
lives in one array compiled into the library, and once warm it must not
take any device memory.  Kept in a file that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from tests.gpu_util import dev_colmajor, dev_vec, host, rel_fro

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5  # the sketch tolerance used by the other GPU tests


def _regular(B, ctx, A, b, n, d, r, seed):
    import torch

    SA = torch.empty((d, r), dtype=torch.float32, device="cuda").t()
    Sb = torch.empty(r, dtype=torch.float32, device="cuda")
    idx = torch.empty(r, dtype=torch.int32, device="cuda")
    B.rnnls_sketch(ctx, A.data_ptr(), A.stride(1), b.data_ptr(), n, d, r, seed, 0, B.RNNLS_SAMPLE_IID,
                   SA.data_ptr(), r, Sb.data_ptr(), idx.data_ptr(), r)
    return SA, Sb, idx


def _noalloc(B, stream, A, b, n, d, r, seed, with_idx=True):
    import torch

    SA = torch.full((d, r), float("nan"), dtype=torch.float32, device="cuda").t()
    Sb = torch.full((r,), float("nan"), dtype=torch.float32, device="cuda")
    idx = torch.full((r,), -1, dtype=torch.int32, device="cuda")
    st = B.lib().rnnls_sketch_noalloc(ctypes.c_void_p(stream), ctypes.c_void_p(A.data_ptr()), A.stride(1),
                                      ctypes.c_void_p(b.data_ptr()), n, d, r, seed, 0,
                                      ctypes.c_void_p(SA.data_ptr()), r, ctypes.c_void_p(Sb.data_ptr()),
                                      ctypes.c_void_p(idx.data_ptr() if with_idx else 0))
    return st, SA, Sb, idx


# the last case is too tall for the sign table to fit the scratch: the kernel then draws D itself
@pytest.mark.parametrize("n,d,r", [((1 << 20) + 77, 9, 4096), (70000, 65, 16384), (3000, 3, 100),
                                   ((1 << 26) + 3, 1, 2000)])
def test_noalloc_matches_regular_sketch_on_two_calls(n, d, r, orc):
    import torch

    from paper_0812_4547_gb300 import _binding as B
    from paper_0812_4547_gb300 import build

    build.build()
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(n + d)
    A_h = rng.standard_normal((n, d)).astype(np.float32)
    b_h = rng.standard_normal(n).astype(np.float32)
    A = dev_colmajor(A_h)
    b = dev_vec(b_h)
    ctx = B.rnnls_create(0, stream)
    try:
        SA0, Sb0, idx0 = _regular(B, ctx, A, b, n, d, r, seed=21)
        torch.cuda.synchronize()
        for call in range(2):
            st, SA1, Sb1, idx1 = _noalloc(B, stream, A, b, n, d, r, seed=21, with_idx=(call == 0))
            assert st == 0, B.rnnls_strerror(st)
            torch.cuda.synchronize()
            if call == 0:
                assert np.array_equal(host(idx1), host(idx0))
            assert rel_fro(host(SA1), host(SA0).astype(np.float64)) <= TOL_F32
            assert rel_fro(host(Sb1), host(Sb0).astype(np.float64)) <= TOL_F32
        # directly against the FP64 oracle on the same FP32 bytes
        idx_ref = orc.sample(21, 0, orc.padded_n(n), r)
        assert np.array_equal(host(idx0), idx_ref)
        if n <= (1 << 21):
            SA_ref, Sb_ref, _ = orc.sketch(A_h, b_h, r, seed=21, instance=0)
            assert rel_fro(host(SA1), SA_ref) <= TOL_F32
            assert rel_fro(host(Sb1), Sb_ref) <= TOL_F32
        else:
            # too tall for a whole oracle sketch in seconds: entries from the
            # definition, to 1e-4 of the entries' typical size sqrt(n/r)
            sc = orc.scale(orc.padded_n(n), r)
            tol = 1e-4 * np.sqrt(n / r)
            got_A, got_b = host(SA1), host(Sb1)
            for k in (0, 1, r // 2, r - 1):
                want_b = orc.sketch_entry(b_h, 21, 0, int(idx_ref[k]), sc)
                assert abs(got_b[k] - want_b) <= tol
                want_a = orc.sketch_entry(A_h[:, 0], 21, 0, int(idx_ref[k]), sc)
                assert abs(got_A[k, 0] - want_a) <= tol
    finally:
        B.rnnls_destroy(ctx)


def test_noalloc_warm_calls_take_no_device_memory():
    """After one warm-up call, further calls leave the device's free memory
    unchanged: no allocation by the library, the runtime or the driver."""
    import torch

    from paper_0812_4547_gb300 import _binding as B

    n, d, r = (1 << 18) + 5, 7, 2048
    rng = np.random.default_rng(5)
    A = dev_colmajor(rng.standard_normal((n, d)), np.float32)
    b = dev_vec(rng.standard_normal(n), np.float32)
    stream = torch.cuda.current_stream().cuda_stream
    SA = torch.empty((d, r), dtype=torch.float32, device="cuda").t()
    Sb = torch.empty(r, dtype=torch.float32, device="cuda")
    idx = torch.empty(r, dtype=torch.int32, device="cuda")
    lib = B.lib()

    def call(seed):
        return lib.rnnls_sketch_noalloc(ctypes.c_void_p(stream), ctypes.c_void_p(A.data_ptr()), A.stride(1),
                                        ctypes.c_void_p(b.data_ptr()), n, d, r, seed, 0,
                                        ctypes.c_void_p(SA.data_ptr()), r, ctypes.c_void_p(Sb.data_ptr()),
                                        ctypes.c_void_p(idx.data_ptr()))

    assert call(1) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for seed in range(2, 6):
        assert call(seed) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_rows_beyond_its_scratch():
    import torch

    from paper_0812_4547_gb300 import _binding as B

    stream = torch.cuda.current_stream().cuda_stream
    A = torch.zeros((2, 1 << 15), dtype=torch.float32, device="cuda").t()
    b = torch.zeros(1 << 15, dtype=torch.float32, device="cuda")
    st, *_ = _noalloc(B, stream, A, b, 1 << 15, 2, 16385, seed=1)
    assert st == B.RNNLS_EUNSUPPORTED
    st, *_ = _noalloc(B, stream, A, b, 1 << 15, 2, 0, seed=1)
    assert st == B.RNNLS_EINVAL
