"""rnnls_solve_pg: the iterative solver on the quadratic-programming form of
Sec. 3.4 (accelerated projected gradient on the equilibrated Q~, q~).

Its result is the unique minimiser to within its stated residual, so it is
compared with the exact Lawson-Hanson solution of the oracle (d <= 200) and,
for d beyond the active-set solve's limit, with a problem whose exact
solution is known: a support P, x_P > 0, and a residual that is orthogonal
to the columns of P and strictly negatively correlated with every other
column, so the KKT conditions pin the minimiser (checked here in FP64 on the
FP32 bytes)."""
import numpy as np
import pytest

from tests.gpu_util import dev_colmajor, dev_vec, host


def kkt_problem(seed, r, d, frac=0.5):
    """(SA, Sb, x) with x the exact NNLS minimiser of the FP32 data."""
    rng = np.random.default_rng(seed)
    SA = rng.standard_normal((r, d)).astype(np.float32)
    P = np.sort(rng.permutation(d)[: int(frac * d)])
    off = np.setdiff1d(np.arange(d), P)
    SP = SA[:, P].astype(np.float64)
    n = rng.standard_normal(r)
    e = n - SP @ np.linalg.lstsq(SP, n, rcond=None)[0]  # orthogonal to the columns of P
    en = e / np.linalg.norm(e)
    for j in off:
        y = rng.standard_normal(r)
        y -= (y @ en) * en
        SA[:, j] = (y - 2.0 * en).astype(np.float32)  # w_j = -2 ||e|| < 0
    xP = rng.uniform(0.5, 2.0, P.size)
    Sb = (SA[:, P].astype(np.float64) @ xP + e).astype(np.float32)
    # the minimiser of the FP32 data: least squares on P, then the KKT conditions
    x = np.zeros(d)
    x[P] = np.linalg.lstsq(SA[:, P].astype(np.float64), Sb.astype(np.float64), rcond=None)[0]
    w = SA.astype(np.float64).T @ (Sb.astype(np.float64) - SA.astype(np.float64) @ x)
    assert np.all(x[P] > 0.1)
    assert np.all(w[off] < -np.linalg.norm(e))  # strict complementarity with a wide margin
    return SA, Sb, x


@pytest.mark.parametrize("seed", [0, 1])
def test_kkt_construction_matches_the_oracle(orc, seed):
    SA, Sb, x = kkt_problem(seed, 300, 40)
    xo, info = orc.nnls(SA, Sb)
    assert info["status"] == 0
    assert np.array_equal(xo > 0, x > 0)
    assert np.max(np.abs(xo - x)) <= 1e-10 * np.max(x)


def _termdoc_sketch(orc, n, d, r, seed):
    import workloads

    p = workloads.problem(2, n=n, d=d, r=r, seed=seed)
    SA, Sb, _ = orc.sketch(p.A.astype(np.float32), p.b.astype(np.float32), r, seed=seed)
    return SA.astype(np.float32), Sb.astype(np.float32)


@pytest.mark.gpu
@pytest.mark.parametrize("n,d,r", [(1 << 13, 20, 512), (1 << 15, 64, 4096), (1 << 14, 200, 4096)])
def test_pg_matches_the_oracle_on_sketches(orc, n, d, r):
    import paper_0812_4547_gb300 as P

    SA, Sb = _termdoc_sketch(orc, n, d, r, seed=d)
    x_ref, info_ref = orc.nnls(SA, Sb)
    ctx = P.Context(0)
    try:
        x, info = ctx.solve_pg(dev_colmajor(SA), dev_vec(Sb), tol=1e-12)
        x_lh, _ = ctx.solve(dev_colmajor(SA), dev_vec(Sb))
        got = P.info_dict(info)
        xg, xl = host(x), host(x_lh)
    finally:
        ctx.close()
    assert got["status"] == 0, got
    scale = np.max(np.abs(x_ref))
    assert np.max(np.abs(xg - x_ref)) <= 1e-6 * scale
    # objective ||SA x - Sb||^2 against the oracle's minimum
    S64, s64 = SA.astype(np.float64), Sb.astype(np.float64)
    f = lambda v: float(np.sum((S64 @ v - s64) ** 2))  # noqa: E731
    assert f(xg) - f(x_ref) <= 1e-10 * f(x_ref)
    assert abs(got["objective"] - f(xg)) <= 1e-9 * f(xg)
    # the large entries agree with the exact support; the GPU active-set solve agrees too
    big = x_ref > 1e-6 * scale
    assert np.all(xg[big] > 0)
    assert np.max(np.abs(xg - xl)) <= 1e-6 * scale


@pytest.mark.gpu
@pytest.mark.parametrize("r,d", [(600, 300), (3000, 1500), (4096, 2048)])
def test_pg_large_d_against_the_kkt_solution(r, d):
    import paper_0812_4547_gb300 as P

    SA, Sb, x_star = kkt_problem(d, r, d)
    ctx = P.Context(0)
    try:
        x, info = ctx.solve_pg(dev_colmajor(SA), dev_vec(Sb), tol=1e-12)
        got = P.info_dict(info)
        xg = host(x)
    finally:
        ctx.close()
    assert got["status"] == 0, got
    assert np.array_equal(xg > 0, x_star > 0)
    assert got["passive_count"] == int(np.count_nonzero(x_star))
    assert np.max(np.abs(xg - x_star)) <= 1e-6 * np.max(x_star)
    assert got["dual_max"] < 0


@pytest.mark.gpu
def test_pg_edge_cases():
    import ctypes

    import torch

    import paper_0812_4547_gb300 as P
    from paper_0812_4547_gb300 import _binding as B

    rng = np.random.default_rng(3)
    ctx = P.Context(0)
    try:
        # b in the negative cone of every column: x = 0
        SA = np.abs(rng.standard_normal((200, 7))).astype(np.float32)
        Sb = -np.abs(rng.standard_normal(200)).astype(np.float32)
        x, info = ctx.solve_pg(dev_colmajor(SA), dev_vec(Sb))
        assert np.all(host(x) == 0.0) and P.info_dict(info)["status"] == 0
        # a NaN in SA: ENONFINITE, x = 0
        SA2 = rng.standard_normal((100, 5)).astype(np.float32)
        SA2[17, 3] = np.nan
        x, info = ctx.solve_pg(dev_colmajor(SA2), dev_vec(rng.standard_normal(100).astype(np.float32)))
        assert P.info_dict(info)["status"] == B.RNNLS_ENONFINITE and np.all(host(x) == 0.0)
        # an iteration cap that is too small: EMAXITER with the iterate so far
        SA3, Sb3 = rng.standard_normal((500, 60)).astype(np.float32), rng.standard_normal(500).astype(np.float32)
        x, info = ctx.solve_pg(dev_colmajor(SA3), dev_vec(Sb3), tol=1e-14, max_iter=3)
        got = P.info_dict(info)
        assert got["status"] == B.RNNLS_EMAXITER and got["outer_iters"] == 3
        assert np.all(host(x) >= 0.0)
        # argument errors
        d = 10
        A = torch.zeros((d, 50), device="cuda").t()
        b = torch.zeros(50, device="cuda")
        xo = torch.zeros(d, dtype=torch.float64, device="cuda")
        lib = B.lib()
        call = lambda dd, tol, it: lib.rnnls_solve_pg(  # noqa: E731
            ctypes.c_void_p(ctx.handle), ctypes.c_void_p(A.data_ptr()), 50, ctypes.c_void_p(b.data_ptr()), 50, dd,
            ctypes.c_void_p(xo.data_ptr()), None, tol, it)
        assert call(d, 0.0, 10) == B.RNNLS_EINVAL
        assert call(d, 1e-9, 0) == B.RNNLS_EINVAL
        assert call(8193, 1e-9, 10) == B.RNNLS_EUNSUPPORTED
    finally:
        ctx.close()
