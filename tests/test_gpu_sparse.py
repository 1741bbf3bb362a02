"""rnnls_sketch_csc: the sketch of Alg. 1 for a sparse A held by columns
(the paper's term-document data are sparse, Sec. 4.1-4.2), against the FP64
oracle's sketch of the same matrix written out densely, and against the
dense GPU sketch (same rows, signs and scale)."""
import numpy as np
import pytest

from tests.gpu_util import dev_colmajor, dev_vec, host, rel_fro

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5


def sparse_matrix(n, d, density, seed, empty_cols=(), full_cols=()):
    rng = np.random.default_rng(seed)
    A = np.where(rng.random((n, d)) < density, np.abs(rng.standard_normal((n, d))), 0.0).astype(np.float32)
    for j in empty_cols:
        A[:, j] = 0.0
    for j in full_cols:
        A[:, j] = rng.standard_normal(n).astype(np.float32)
    return A


def to_device_csc(A):
    """colptr (int64), rowidx (int32, ascending per column), val (float32) on the device."""
    import torch

    n, d = A.shape
    rows, vals, ptr = [], [], [0]
    for j in range(d):
        nz = np.flatnonzero(A[:, j])
        rows.append(nz.astype(np.int32))
        vals.append(A[nz, j].astype(np.float32))
        ptr.append(ptr[-1] + nz.size)
    rowidx = np.concatenate(rows) if ptr[-1] else np.zeros(0, np.int32)
    val = np.concatenate(vals) if ptr[-1] else np.zeros(0, np.float32)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    return to(np.asarray(ptr, np.int64)), to(rowidx), to(val)


def _both(ctx, A, b, r, seed):
    import torch

    n, d = A.shape
    colptr, rowidx, val = to_device_csc(A)
    bd = dev_vec(b)
    SA, Sb, idx = ctx.sketch_csc(colptr, rowidx, val, bd, n, d, r, seed)
    SA2 = torch.empty((d, r), dtype=torch.float32, device="cuda").t()
    Sb2 = torch.empty(r, dtype=torch.float32, device="cuda")
    idx2 = torch.empty(r, dtype=torch.int32, device="cuda")
    ctx.sketch(dev_colmajor(A), bd, r, seed=seed, SA=SA2, Sb=Sb2, idx=idx2, want_count=False)
    torch.cuda.synchronize()
    return host(SA), host(Sb), host(idx), host(SA2), host(Sb2), host(idx2)


@pytest.mark.parametrize("n,d,r,density,empty,full", [
    (10000, 300, 350, 0.02, (5,), ()),       # Sec. 4.2's size at 2 % density
    (10000, 300, 450, 0.64, (), (7,)),       # ... and at 64 %
    (4096, 3, 100, 0.05, (1,), (2,)),        # one chunk per step
    (8192 - 5, 17, 1000, 0.02, (), ()),      # two chunks per step, ragged
    (70001, 33, 16384, 0.02, (0, 32), ()),   # the largest r
])
def test_csc_sketch_matches_oracle_and_dense(orc, n, d, r, density, empty, full):
    import paper_0812_4547_gb300 as P

    A = sparse_matrix(n, d, density, seed=n + d, empty_cols=empty, full_cols=full)
    b = np.random.default_rng(d).standard_normal(n).astype(np.float32)
    ctx = P.Context(0)
    try:
        SA, Sb, idx, SA2, Sb2, idx2 = _both(ctx, A, b, r, seed=11)
    finally:
        ctx.close()
    SA_ref, Sb_ref, idx_ref = orc.sketch(A, b, r, seed=11)
    assert np.array_equal(idx, idx_ref) and np.array_equal(idx2, idx_ref)
    assert rel_fro(SA, SA_ref) <= TOL_F32 and rel_fro(Sb, Sb_ref) <= TOL_F32
    for j in empty:
        assert np.all(SA[:, j] == 0.0)
    assert rel_fro(SA, SA2.astype(np.float64)) <= TOL_F32


def test_csc_sketch_tall(orc):
    """2^20 + 77 rows at 2 %: entries from the definition (oracle), and the
    dense GPU sketch of the same matrix."""
    import paper_0812_4547_gb300 as P

    n, d, r = (1 << 20) + 77, 9, 4096
    A = sparse_matrix(n, d, 0.02, seed=3)
    b = np.random.default_rng(4).standard_normal(n).astype(np.float32)
    ctx = P.Context(0)
    try:
        SA, Sb, idx, SA2, Sb2, idx2 = _both(ctx, A, b, r, seed=5)
    finally:
        ctx.close()
    assert np.array_equal(idx, idx2)
    assert rel_fro(SA, SA2.astype(np.float64)) <= TOL_F32 and rel_fro(Sb, Sb2.astype(np.float64)) <= TOL_F32
    sc = orc.scale(orc.padded_n(n), r)
    for k in (0, 7, r // 2, r - 1):
        for j in (0, d - 1):
            want = orc.sketch_entry(A[:, j], 5, 0, int(idx[k]), sc)
            assert abs(SA[k, j] - want) <= 1e-4 * np.sqrt(n / r) * np.sqrt(0.02)
        want_b = orc.sketch_entry(b, 5, 0, int(idx[k]), sc)
        assert abs(Sb[k] - want_b) <= 1e-4 * np.sqrt(n / r)


def test_csc_sketch_refusals():
    import torch

    import paper_0812_4547_gb300 as P
    from paper_0812_4547_gb300 import _binding as B

    ctx = P.Context(0)
    try:
        A = sparse_matrix(5000, 2, 0.1, seed=1)
        colptr, rowidx, val = to_device_csc(A)
        b = torch.zeros(5000, device="cuda")
        with pytest.raises(B.RNNLSError) as e:
            ctx.sketch_csc(colptr, rowidx, val, b, 5000, 2, 16385, 1)
        assert e.value.status == B.RNNLS_EUNSUPPORTED
        A2 = sparse_matrix(2048, 2, 0.1, seed=2)
        c2, r2, v2 = to_device_csc(A2)
        with pytest.raises(B.RNNLSError) as e:
            ctx.sketch_csc(c2, r2, v2, torch.zeros(2048, device="cuda"), 2048, 2, 10, 1)
        assert e.value.status == B.RNNLS_EUNSUPPORTED
    finally:
        ctx.close()
