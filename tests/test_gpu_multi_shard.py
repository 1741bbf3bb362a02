"""GPU parity of the multi-target sketch and of the row-shard sketch.

rnnls_sketch_multi applies one S H D to [A | B]: every target column must
match the oracle's sketch of (A, B[:, t]) with the same seed, and the
one-target case must equal rnnls_sketch exactly.  rnnls_sketch_shard gives
a row block's part of the sketch: the parts of any split into blocks that
start on 16384-row boundaries must add up to the full sketch.
"""
import numpy as np
import pytest

from tests.gpu_util import dev_colmajor, dev_vec, host, rel_fro

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5  # FP32 sketch vs the FP64 oracle on the same FP32 bytes
TOL_SUM = 1e-6  # sum of shard parts vs the one-piece FP32 sketch (different summation order)


@pytest.fixture(scope="module")
def ctx():
    import paper_0812_4547_gb300 as P

    c = P.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("n,d,nrhs,r", [(5000, 3, 4, 300), ((1 << 16) + 5, 6, 5, 700), (300000, 20, 33, 5000),
                                        (1 << 18, 2, 3, 12000)])
def test_sketch_multi_matches_oracle_per_target(ctx, orc, n, d, nrhs, r):
    rng = np.random.default_rng(n + nrhs)
    A = rng.standard_normal((n, d)).astype(np.float32)
    Bm = rng.random((n, nrhs)).astype(np.float32)
    SA, SB, idx = ctx.sketch_multi(dev_colmajor(A), dev_colmajor(Bm), r, seed=5, instance=1)
    SA, SB, idx = host(SA), host(SB), host(idx)
    for t in sorted({0, nrhs // 2, nrhs - 1}):
        SA_o, Sb_o, idx_o = orc.sketch(A.astype(np.float64), Bm[:, t].astype(np.float64), r, 5, 1)
        assert np.array_equal(idx, idx_o)
        assert rel_fro(SA, SA_o) <= TOL_F32
        assert rel_fro(SB[:, t], Sb_o) <= TOL_F32


@pytest.mark.parametrize("n", [3000, (1 << 17) + 77])
def test_sketch_multi_one_target_is_the_plain_sketch(ctx, n):
    rng = np.random.default_rng(n)
    A = dev_colmajor(rng.standard_normal((n, 7)), np.float32)
    b = rng.standard_normal(n).astype(np.float32)
    SA1, Sb1, idx1, _ = ctx.sketch(A, dev_vec(b), 2048, seed=9, instance=3)
    SA2, SB2, idx2 = ctx.sketch_multi(A, dev_colmajor(b[:, None]), 2048, seed=9, instance=3)
    assert np.array_equal(host(idx1), host(idx2))
    assert np.array_equal(host(SA1), host(SA2))
    assert np.array_equal(host(Sb1), host(SB2)[:, 0])


def _bounds(n: int, parts: int):
    """Row blocks of the padded n starting on multiples of 16384 (uneven when they must be)."""
    groups = n // 16384
    cuts = [round(g * groups / parts) * 16384 for g in range(parts + 1)]
    return [(cuts[g], cuts[g + 1] - cuts[g]) for g in range(parts) if cuts[g + 1] > cuts[g]]


@pytest.mark.parametrize("n_raw,d,r,parts", [((1 << 18) + 1000, 5, 3000, 2), ((1 << 18) + 1000, 5, 3000, 4),
                                             (200000, 8, 5000, 3), (1 << 17, 3, 700, 8)])
def test_shard_parts_add_up_to_the_sketch(ctx, orc, n_raw, d, r, parts):
    import torch

    rng = np.random.default_rng(n_raw + parts)
    A = rng.standard_normal((n_raw, d)).astype(np.float32)
    b = rng.standard_normal(n_raw).astype(np.float32)
    SA_full, Sb_full, idx_full, _ = ctx.sketch(dev_colmajor(A), dev_vec(b), r, seed=13, instance=2)
    n = orc.padded_n(n_raw)
    SA_sum = torch.zeros((r, d), dtype=torch.float64, device="cuda")
    Sb_sum = torch.zeros(r, dtype=torch.float64, device="cuda")
    for row0, rows in _bounds(n, parts):
        v = max(0, min(rows, n_raw - row0))
        A_rows = dev_colmajor(A[row0:row0 + v] if v else np.zeros((1, d), np.float32))
        b_rows = dev_vec(b[row0:row0 + v] if v else np.zeros(1, np.float32))
        SA_g, Sb_g, idx_g = ctx.sketch_shard(A_rows, b_rows, n_raw, row0, r, seed=13, instance=2)
        assert np.array_equal(host(idx_g), host(idx_full))
        SA_sum += SA_g.double()
        Sb_sum += Sb_g.double()
    assert rel_fro(host(SA_sum), host(SA_full).astype(np.float64)) <= TOL_SUM
    assert rel_fro(host(Sb_sum), host(Sb_full).astype(np.float64)) <= TOL_SUM
    SA_o, Sb_o, _ = orc.sketch(A.astype(np.float64), b.astype(np.float64), r, 13, 2)
    assert rel_fro(host(SA_sum), SA_o) <= TOL_F32
    assert rel_fro(host(Sb_sum), Sb_o) <= TOL_F32


def test_shard_rejects_unaligned_start(ctx):
    import paper_0812_4547_gb300 as P

    A = dev_colmajor(np.ones((20000, 2)), np.float32)
    b = dev_vec(np.ones(20000), np.float32)
    with pytest.raises(P.RNNLSError):
        ctx.sketch_shard(A, b, 1 << 16, 1000, 100, seed=1)


def _infos(raw):
    import paper_0812_4547_gb300 as P

    return [P.info_dict(raw[t]) for t in range(raw.shape[0])]


@pytest.mark.parametrize("m,d,nrhs,seed", [(300, 5, 7, 0), (4096, 64, 40, 1), (2000, 100, 256, 2), (8192, 128, 3, 3)])
def test_solve_multi_matches_oracle_per_target(ctx, orc, m, d, nrhs, seed):
    """Every target's Lawson-Hanson solve on the shared sketch: identical passive set, x within 1e-6."""
    rng = np.random.default_rng(seed)
    S = rng.standard_normal((m, d)).astype(np.float32)
    Xt = np.maximum(rng.standard_normal((d, nrhs)), 0) * (rng.random((d, nrhs)) < 0.5)
    SB = (S.astype(np.float64) @ Xt + 0.1 * rng.standard_normal((m, nrhs))).astype(np.float32)
    X, raw = ctx.solve_multi(dev_colmajor(S), dev_colmajor(SB))
    X = host(X)
    infos = _infos(raw)
    for t in sorted({0, 1 % nrhs, nrhs // 2, nrhs - 1}):
        xo, io = orc.nnls(S.astype(np.float64), SB[:, t].astype(np.float64))
        assert infos[t]["status"] == io["status"] == 0, (t, infos[t], io)
        assert np.array_equal(X[:, t] > 0, xo > 0), t
        assert np.linalg.norm(X[:, t] - xo) / max(np.linalg.norm(xo), 1e-300) <= 1e-6
        assert infos[t]["passive_count"] == io["passive_count"]
    assert all(inf["status"] == 0 for inf in infos)


def test_multi_target_pipeline_end_to_end(ctx, orc):
    """Workload-4 shape at reduced size: one sketch of [A | B], one shared Gram, per-target solves,
    each equal to the single-target path of the same seed."""
    A, Bm, _ = workloads_multi(n=1 << 16, d=20, nrhs=12)
    SA, SB, idx = ctx.sketch_multi(dev_colmajor(A, np.float32), dev_colmajor(Bm, np.float32), 1024, seed=3, instance=0)
    X, raw = ctx.solve_multi(SA, SB)
    X = host(X)
    for t in (0, 5, 11):
        SA1, Sb1, _, _ = ctx.sketch(dev_colmajor(A, np.float32), dev_vec(Bm[:, t], np.float32), 1024, seed=3, instance=0)
        x1, _ = ctx.solve(SA1, Sb1)
        x1 = host(x1)
        assert np.array_equal(X[:, t] > 0, x1 > 0)
        assert np.linalg.norm(X[:, t] - x1) / max(np.linalg.norm(x1), 1e-300) <= 1e-6


def workloads_multi(n, d, nrhs):
    import workloads

    return workloads.multi_rhs(n=n, d=d, nrhs=nrhs, r=1024)[:3]


def test_sketch_multi_full_size_sampled_entries(ctx, orc):
    """Workload 4's sizes (A 2^20 x 100, B 2^20 x 256, r = 4096) in the
    benchmark's launch configuration: rows bit-exact, sampled entries of A's
    and B's sketches against the definition (O(n) each)."""
    import math

    import paper_0812_4547_gb300 as P

    n, d, nrhs, r = 1 << 20, 100, 256, 4096
    rng = np.random.default_rng(44)
    A = rng.random((n, d), dtype=np.float32)
    Bm = rng.random((n, nrhs), dtype=np.float32)
    SA, SB, idx = ctx.sketch_multi(dev_colmajor(A), dev_colmajor(Bm), r, seed=9, instance=0)
    idx_o = orc.sample(9, 0, P.padded_n(n), r)
    assert np.array_equal(host(idx), idx_o)
    SAh, SBh = host(SA), host(SB)
    sc = 1 / math.sqrt(r)
    for _ in range(10):
        k = int(rng.integers(r))
        c = int(rng.integers(d + nrhs))
        col = (A[:, c] if c < d else Bm[:, c - d]).astype(np.float64)
        want = orc.sketch_entry(col, 9, 0, int(idx_o[k]), sc)
        got = SAh[k, c] if c < d else SBh[k, c - d]
        assert abs(got - want) <= 1e-5 * sc * np.linalg.norm(col)
