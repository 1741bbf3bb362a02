"""GPU parity of repeated RandomizedNNLS (rnnls_solve_boosted).

Run j of the library must be Alg. 1 with instance instance0 + j: its
sketch is the one rnnls_sketch gives (checked through the oracle's
Lawson-Hanson solve on that sketch), the residuals it reports must match
the FP64 oracle's ||A x_j - b||^2 and the kept run must be the oracle's
choice among them (either of two runs whose residuals agree within the
residual tolerance).
"""
import numpy as np
import pytest

import workloads
from tests.gpu_util import dev_colmajor, dev_vec, host

pytestmark = pytest.mark.gpu

TOL_RES = 1e-6  # FP32 row dot products, FP64 sums of squares
TOL_X = 1e-6    # x on the same sketch, as for rnnls_solve


def _problem(n, d, seed):
    rng = np.random.default_rng(seed)
    A = workloads.termdoc_matrix(n, d, rng, density=0.2).astype(np.float32)
    x = workloads.planted_x(d, d // 2, rng)
    b = workloads.noisy_target(A.astype(np.float64), x, rng, noise_rel=0.1).astype(np.float32)
    return A, b


@pytest.fixture(scope="module")
def ctx():
    import paper_0812_4547_gb300 as P

    c = P.Context(0)
    yield c
    c.close()


def _check_against_oracle(ctx, orc, A, b, A_d, b_d, r, k, seed, inst0):
    import paper_0812_4547_gb300 as P

    import torch

    x, resid, best, info = ctx.solve_boosted(A_d, b_d, r, k, seed, inst0)
    x, resid, best = host(x), host(resid), int(host(best)[0])
    A64, b64 = A.astype(np.float64), b.astype(np.float64)
    # the runs' sketches, by the batched sketch the boosted call uses (the
    # same bits; rnnls_sketch agrees with it to FP32 summation order)
    d = A.shape[1]
    items = [(A_d, b_d, r, seed, inst0 + j, torch.empty((d, r), device="cuda").t(), torch.empty(r, device="cuda"),
              torch.empty(r, dtype=torch.int32, device="cuda")) for j in range(k)]
    ctx.sketch_batched(items)
    res_o, xs_o, ok = [], [], []
    for j in range(k):
        SA, Sb = items[j][5], items[j][6]
        xo, io = orc.nnls(host(SA), host(Sb))
        xs_o.append(xo)
        ok.append(io["status"] == orc.OK)
        res_o.append(orc.residual_sq(A64, b64, xo))
    res_o = np.array(res_o)
    assert np.all(np.abs(resid - res_o) <= TOL_RES * res_o), (resid, res_o)
    cand = [j for j in range(k) if ok[j]]
    if cand:
        m = min(res_o[j] for j in cand)
        assert ok[best] and res_o[best] <= m * (1 + 2 * TOL_RES)
        strict = [j for j in cand if res_o[j] <= m * (1 + 2 * TOL_RES)]
        assert best == min(strict) or len(strict) > 1
    else:
        assert best == 0
    assert np.linalg.norm(x - xs_o[best]) <= TOL_X * max(np.linalg.norm(xs_o[best]), 1e-300)
    if ok[best]:
        assert P.info_dict(info)["status"] == orc.OK
    return best, res_o


@pytest.mark.parametrize("n,d,r,k", [(3 * 16384 + 77, 12, 256, 5), (5000, 6, 64, 3), (70000, 20, 1000, 8),
                                     ((1 << 16), 3, 40, 16)])
def test_boosted_matches_oracle_runs(ctx, orc, n, d, r, k):
    A, b = _problem(n, d, n + d)
    _check_against_oracle(ctx, orc, A, b, dev_colmajor(A), dev_vec(b), r, k, seed=7, inst0=3)


def test_one_run_is_the_plain_algorithm(ctx, orc):
    import torch

    A, b = _problem(40000, 10, 1)
    A_d, b_d = dev_colmajor(A), dev_vec(b)
    x, resid, best, info = ctx.solve_boosted(A_d, b_d, 500, 1, seed=2, instance0=9)
    SA, Sb, _, _ = ctx.sketch(A_d, b_d, 500, seed=2, instance=9)
    x1, _ = ctx.solve(SA, Sb)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    ctx.residual(A_d, b_d, x, out)
    assert int(host(best)[0]) == 0
    # the same run up to the FP32 summation order of the two sketch paths
    assert np.linalg.norm(host(x) - host(x1)) <= 1e-4 * np.linalg.norm(host(x1))
    assert np.array_equal(host(x) > 0, host(x1) > 0)
    assert abs(host(resid)[0] - host(out)[0]) <= TOL_RES * host(out)[0]


def test_full_size_workload_two(ctx):
    """The 2^20 x 64, r = 4096 workload with 4 runs: every run's residual
    against the library's FP64 residual of that run's own solution."""
    import torch

    p = workloads.problem(2)
    A_d = torch.from_numpy(np.ascontiguousarray(p.A.T)).cuda().t()
    b_d = torch.from_numpy(p.b).cuda()
    k = 4
    x, resid, best, info = ctx.solve_boosted(A_d, b_d, p.r, k, seed=0)
    resid = host(resid)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    d = A_d.shape[1]
    items = [(A_d, b_d, p.r, 0, j, torch.empty((d, p.r), device="cuda").t(), torch.empty(p.r, device="cuda"),
              torch.empty(p.r, dtype=torch.int32, device="cuda")) for j in range(k)]
    ctx.sketch_batched(items)
    runs = []
    for j in range(k):
        xj, _ = ctx.solve(items[j][5], items[j][6])
        ctx.residual(A_d, b_d, xj, out)
        runs.append(float(host(out)[0]))
    runs = np.array(runs)
    assert np.all(np.abs(resid - runs) <= TOL_RES * runs)
    bj = int(host(best)[0])
    assert runs[bj] <= runs.min() * (1 + 2 * TOL_RES)


def test_boosted_rejects_bad_arguments(ctx):
    import torch

    import paper_0812_4547_gb300 as P

    A = torch.zeros((3, 20000), device="cuda").t()
    b = torch.zeros(20000, device="cuda")
    with pytest.raises(P.RNNLSError):
        ctx.solve_boosted(A, b, 100, 0, seed=1)
    with pytest.raises(P.RNNLSError):
        ctx.solve_boosted(A, b, 100, 17, seed=1)
    A_wide = torch.zeros((257, 20000), device="cuda").t()
    with pytest.raises(P.RNNLSError):
        ctx.solve_boosted(A_wide, b, 100, 2, seed=1)
