"""GPU parity of the Lawson-Hanson solve (Alg. 1 step 5) against the oracle.

The GPU solve and the oracle solve run on the same sketch bytes (the GPU's
FP32 SA promoted exactly to FP64 for the oracle).  Bar: identical passive
(active) sets, x within 1e-6 relative, same status.
"""
import numpy as np
import pytest

import workloads
from tests.gpu_util import dev_colmajor, dev_vec, host

pytestmark = pytest.mark.gpu

TOL_X = 1e-6


@pytest.fixture(scope="module")
def ctx():
    import paper_0812_4547_gb300 as P

    c = P.Context(0)
    yield c
    c.close()


def solve_both(ctx, orc, S, s, dtype=np.float32):
    import paper_0812_4547_gb300 as P

    S = np.asarray(S, dtype=dtype)
    s = np.asarray(s, dtype=dtype)
    x, info = ctx.solve(dev_colmajor(S), dev_vec(s))
    xg = host(x)
    inf = P.info_dict(info)
    xo, io = orc.nnls(S, s)
    return xg, inf, xo, io


def check_match(xg, inf, xo, io):
    assert inf["status"] == io["status"] == 0, (inf, io)
    assert np.array_equal(xg > 0, xo > 0), (np.nonzero(xg > 0), np.nonzero(xo > 0))
    den = max(np.linalg.norm(xo), 1e-300)
    assert np.linalg.norm(xg - xo) / den <= TOL_X
    assert inf["passive_count"] == io["passive_count"]


@pytest.mark.parametrize("m,d,seed", [(50, 1, 0), (200, 5, 1), (300, 15, 2), (1000, 40, 3), (4096, 64, 4),
                                      (2000, 100, 5), (8192, 128, 6), (4096, 200, 7)])
def test_random_problems(ctx, orc, m, d, seed):
    rng = np.random.default_rng(seed)
    S = rng.standard_normal((m, d))
    s = rng.standard_normal(m) + S @ np.maximum(rng.standard_normal(d), 0)
    check_match(*solve_both(ctx, orc, S, s))


@pytest.mark.parametrize("d,r", [(16, 512), (64, 4096), (128, 8192)])
def test_sketch_of_termdoc_workload(ctx, orc, d, r):
    # the oracle's own sketch of a term-document problem, solved on both sides
    p = workloads.problem(2, n=1 << 15, d=d, r=r)
    SA, Sb, _ = orc.sketch(p.A, p.b, r, seed=1)
    check_match(*solve_both(ctx, orc, SA.astype(np.float32), Sb.astype(np.float32)))


def test_interpolation_steps(ctx, orc):
    # nearly low-rank columns force many interpolation (alpha) steps
    for seed in range(6):
        rng = np.random.default_rng(300 + seed)
        S = rng.standard_normal((40, 3)) @ rng.standard_normal((3, 15)) + 0.1 * rng.standard_normal((40, 15))
        s = rng.standard_normal(40)
        xg, inf, xo, io = solve_both(ctx, orc, S, s)
        check_match(xg, inf, xo, io)
        assert inf["outer_iters"] == io["outer_iters"]
        assert inf["inner_iters"] == io["inner_iters"]


def test_degenerate(ctx, orc):
    rng = np.random.default_rng(1)
    S = rng.random((100, 6))
    xg, inf, xo, io = solve_both(ctx, orc, S, np.zeros(100))
    assert np.all(xg == 0) and inf["passive_count"] == 0 and inf["status"] == 0
    xg, inf, xo, io = solve_both(ctx, orc, S, -S.sum(axis=1))
    assert np.all(xg == 0)
    xg, inf, xo, io = solve_both(ctx, orc, S[:, :1], 3 * S[:, 0])
    assert abs(xg[0] - 3.0) < 1e-6


def test_info_fields(ctx, orc):
    rng = np.random.default_rng(2)
    S = rng.random((500, 12))
    s = rng.random(500)
    xg, inf, xo, io = solve_both(ctx, orc, S, s)
    S64 = S.astype(np.float32).astype(np.float64)
    s64 = s.astype(np.float32).astype(np.float64)
    assert inf["tol"] == pytest.approx(orc.lh_tol(S64, s64), rel=1e-6)
    obj = np.linalg.norm(S64 @ xo - s64) ** 2
    assert inf["objective"] == pytest.approx(obj, rel=1e-8)
    assert inf["dual_max"] <= inf["tol"]


def test_fp64_solve(ctx, orc):
    p = workloads.problem(1)
    SA, Sb, _ = orc.sketch(p.A, p.b, p.r, seed=0)
    xg, inf, xo, io = solve_both(ctx, orc, SA, Sb, dtype=np.float64)
    check_match(xg, inf, xo, io)


def test_batched_uneven(ctx, orc):
    import torch

    import paper_0812_4547_gb300 as P

    rng = np.random.default_rng(3)
    probs, want = [], []
    for i, (m, d) in enumerate([(300, 10), (1000, 50), (77, 3), (4096, 120), (512, 64)]):
        S = rng.standard_normal((m, d)).astype(np.float32)
        s = (rng.standard_normal(m) + S @ np.maximum(rng.standard_normal(d), 0)).astype(np.float32)
        x = torch.empty(d, dtype=torch.float64, device="cuda")
        info = torch.zeros(P.INFO_BYTES, dtype=torch.uint8, device="cuda")
        probs.append((dev_colmajor(S), dev_vec(s), x, info))
        want.append(orc.nnls(S, s))
    ctx.solve_batched(probs)
    torch.cuda.synchronize()
    for (SA, Sb, x, info), (xo, io) in zip(probs, want):
        check_match(host(x), P.info_dict(info), xo, io)


def test_residual(ctx, orc):
    rng = np.random.default_rng(4)
    A = rng.random((100000, 7)).astype(np.float32)
    b = rng.random(100000).astype(np.float32)
    x = rng.random(7)
    out = ctx.residual(dev_colmajor(A), dev_vec(b), dev_vec(x))
    assert host(out)[0] == pytest.approx(orc.residual_sq(A, b, x), rel=1e-12)


def test_end_to_end_randomized_nnls(ctx, orc):
    # sketch + solve on device vs the all-FP64 oracle pipeline: the sketch
    # differs at FP32 rounding, so x~ agrees to the conditioning of the
    # small problem; the residual ratio of Theorem 1 is compared directly.
    p = workloads.problem(2, n=1 << 16, d=32, r=2048)
    x, info, _ = ctx.randomized_nnls(dev_colmajor(p.A), dev_vec(p.b), p.r, seed=5)
    xg = host(x)
    xo, io, _ = orc.randomized_nnls(p.A, p.b, p.r, 5)
    xopt, _ = orc.exact_nnls(p.A, p.b)
    opt = orc.residual_sq(p.A, p.b, xopt)
    rg = orc.residual_sq(p.A, p.b, xg) / opt
    ro = orc.residual_sq(p.A, p.b, xo) / opt
    assert rg >= 1 - 1e-9
    assert abs(rg - ro) <= 1e-6 * ro
    assert np.linalg.norm(xg - xo) <= 1e-3 * np.linalg.norm(xo)


# d above about 230: the passive-block inverse no longer fits in shared
# memory and is kept in the workspace (one block per solve either way)
@pytest.mark.parametrize("m,d,seed", [(450, 300, 11), (1200, 600, 12)])
def test_large_d(ctx, orc, m, d, seed):
    rng = np.random.default_rng(seed)
    S = rng.standard_normal((m, d))
    s = rng.standard_normal(m) + S @ np.maximum(rng.standard_normal(d), 0)
    check_match(*solve_both(ctx, orc, S, s))


def test_large_d_batched_and_multi(ctx, orc):
    import torch

    import paper_0812_4547_gb300 as P

    rng = np.random.default_rng(21)
    shapes = [(400, 300), (300, 40), (700, 500)]
    probs, data = [], []
    for m, d in shapes:
        S = rng.standard_normal((m, d)).astype(np.float32)
        s = (rng.standard_normal(m) + S @ np.maximum(rng.standard_normal(d), 0)).astype(np.float32)
        x = torch.empty(d, dtype=torch.float64, device="cuda")
        info = torch.zeros(P.INFO_BYTES, dtype=torch.uint8, device="cuda")
        probs.append((dev_colmajor(S), dev_vec(s), x, info))
        data.append((S, s))
    ctx.solve_batched(probs)
    torch.cuda.synchronize()
    for (S, s), (_, _, x, info) in zip(data, probs):
        xo, io = orc.nnls(S, s)
        check_match(host(x), P.info_dict(info), xo, io)
    # three targets sharing one sketch with d = 300
    m, d, nrhs = 450, 300, 3
    S = rng.standard_normal((m, d)).astype(np.float32)
    T = np.stack([rng.standard_normal(m) + S @ np.maximum(rng.standard_normal(d), 0) for _ in range(nrhs)],
                 axis=1).astype(np.float32)
    X, infos = ctx.solve_multi(dev_colmajor(S), dev_colmajor(T), r=m)
    X = host(X)
    for t in range(nrhs):
        xo, io = orc.nnls(S, T[:, t])
        check_match(X[:, t], P.info_dict(infos[t]), xo, io)


def test_d_beyond_the_limit_is_refused(ctx):
    import torch

    import paper_0812_4547_gb300 as P

    S = torch.zeros((1025, 1100), device="cuda").t()
    s = torch.zeros(1100, device="cuda")
    with pytest.raises(P.RNNLSError):
        ctx.solve(S, s)


def test_batched_solve_of_workload_five_sketches(ctx, orc):
    """Workload 5's solve at its real sizes (r up to 32768, d up to 200): the
    batched sketch of term-document instances, then the batched solve; every
    x against the oracle's Lawson-Hanson on the same sketch bytes."""
    import torch

    import bench
    import paper_0812_4547_gb300 as P

    shapes = [(1 << 18, 200, 32768), (1 << 17, 150, 16384), (50000, 60, 8192), (20000, 16, 2048)]
    insts = bench.device_batch(shapes, 7, torch.device("cuda"))
    items, probs = [], []
    for i, (A, b, r) in enumerate(insts):
        d = A.shape[1]
        SA = torch.empty((d, r), device="cuda").t()
        Sb = torch.empty(r, device="cuda")
        items.append((A, b, r, 3, i, SA, Sb, torch.empty(r, dtype=torch.int32, device="cuda")))
        x = torch.empty(d, dtype=torch.float64, device="cuda")
        info = torch.zeros(P.INFO_BYTES, dtype=torch.uint8, device="cuda")
        probs.append((SA, Sb, x, info))
    ctx.sketch_batched(items)
    ctx.solve_batched(probs)
    torch.cuda.synchronize()
    for SA, Sb, x, info in probs:
        xo, io = orc.nnls(host(SA), host(Sb))
        check_match(host(x), P.info_dict(info), xo, io)
