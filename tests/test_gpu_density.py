"""The density experiment's inputs and one of its problems (Sec. 4.2).

The generator must give the stated density with non-zeros in (0, 1]; one
problem at d = 300 goes through the library (sketch, Lawson-Hanson on the
sketch, Lawson-Hanson on the full A) and its relative error
||A x~ - b|| / ||A x_opt - b|| must match the FP64 oracle's on the same
sketch and the same full data.
"""
import math

import numpy as np
import pytest

from tests.gpu_util import host

pytestmark = pytest.mark.gpu


def test_density_matrix_statistics():
    import torch

    import bench

    X = bench.density_matrix(10000, 301, 0.08, seed=5, dev=torch.device("cuda"))
    Xh = host(X)
    assert Xh.shape == (10000, 301)
    frac = np.count_nonzero(Xh) / Xh.size
    assert abs(frac - 0.08) < 0.003
    nz = Xh[Xh != 0]
    assert nz.min() > 0 and nz.max() <= 1.0


def test_one_density_problem_matches_oracle(orc):
    import torch

    import bench
    import paper_0812_4547_gb300 as P

    n, d, r = 10000, 300, 350
    X = bench.density_matrix(n, d + 1, 0.16, seed=11, dev=torch.device("cuda"))
    A = X[:, 1:].contiguous().t().contiguous().t()
    b = X[:, 0].contiguous()
    ctx = P.Context(0)
    try:
        x_opt, _ = ctx.solve(A, b, r=n)
        x, info, (SA, Sb, _, rows) = ctx.randomized_nnls(A, b, r, seed=3)
        res_g = float(ctx.residual(A, b, x).item())
        res_og = float(ctx.residual(A, b, x_opt).item())
    finally:
        ctx.close()
    Ah, bh = host(A).astype(np.float64), host(b).astype(np.float64)
    xo_sk, io = orc.nnls(host(SA)[:rows], host(Sb)[:rows])
    xo_opt, io2 = orc.nnls(Ah, bh)
    assert io["status"] == io2["status"] == 0
    assert np.linalg.norm(host(x) - xo_sk) <= 1e-6 * np.linalg.norm(xo_sk)
    assert np.linalg.norm(host(x_opt) - xo_opt) <= 1e-6 * np.linalg.norm(xo_opt)
    rel_g = math.sqrt(res_g / res_og)
    rel_o = math.sqrt(orc.residual_sq(Ah, bh, xo_sk) / orc.residual_sq(Ah, bh, xo_opt))
    assert rel_o >= 1.0 - 1e-12
    assert abs(rel_g - rel_o) <= 1e-6 * rel_o
