"""The Lawson-Hanson solve's switch to its accurate mode (Sec. 2.2's
active-set method, every step refined in float-float) made to happen.

The problems have a near-tie: at the optimum over a support P, one inactive
column j0 has a dual w_j0 = 30 tol or 5 tol -- clearly positive in FP64, yet
within the noise of an FP32 dual (about 10 to 20 tol on these sizes) -- and
every other inactive column a strongly negative one.  The exact method
therefore adds j0 with a tiny positive value.  The solver's FP32 iterations
miss j0 in some of the problems (rarely at 30 tol, often at 5 tol); their
end-point check in float-float then finds w_j0 > tol and continues in the
accurate mode (info.accurate_mode = 2).  Either way the final active set must
be the oracle's and x within 1e-6 of it."""
import numpy as np
import pytest

from tests.gpu_util import dev_colmajor, dev_vec, host


def near_tie_problem(orc, seed, r=2000, d=40, npass=15, delta_tols=30.0, dependent=0.0):
    """SA (r x d) and Sb (FP32) whose NNLS optimum is P = {0..npass-1} plus
    j0, entering with dual delta_tols * tol at the optimum over P.  With
    dependent > 0, column 1 is column 0 plus that much noise (cond(Q) grows
    like 1 / dependent^2)."""
    rng = np.random.default_rng(seed)
    SA = rng.standard_normal((r, d)).astype(np.float32)
    if dependent > 0:
        SA[:, 1] = (SA[:, 0] + dependent * rng.standard_normal(r)).astype(np.float32)
    P = np.arange(npass)
    x_P = rng.uniform(0.5, 2.0, npass)
    Sb = (SA[:, P].astype(np.float64) @ x_P + rng.standard_normal(r)).astype(np.float32)
    xs, *_ = np.linalg.lstsq(SA[:, P].astype(np.float64), Sb.astype(np.float64), rcond=None)
    e = Sb.astype(np.float64) - SA[:, P].astype(np.float64) @ xs  # residual at the optimum over P
    en = e / np.linalg.norm(e)
    j0 = npass + int(rng.integers(0, d - npass))
    for j in range(npass, d):
        y = rng.standard_normal(r)
        y = y - (y @ en) * en
        if j != j0:
            y = y - 3.0 * en  # w_j = y'e = -3 ||e||
        SA[:, j] = y.astype(np.float32)
    delta = delta_tols * orc.lh_tol(SA, Sb)
    # w_j0 = delta: a Newton step on the entry where the residual is largest,
    # repeated until the FP32 column holds it
    y = SA[:, j0].astype(np.float64)
    k = int(np.argmax(np.abs(e)))
    for _ in range(3):
        y[k] -= (y @ e - delta) / e[k]
        y = y.astype(np.float32).astype(np.float64)
    SA[:, j0] = y.astype(np.float32)
    return SA, Sb, j0


@pytest.mark.parametrize("seed,delta_tols", [(0, 30.0), (3, 30.0), (6, 30.0), (200, 5.0), (207, 5.0), (211, 5.0)])
def test_construction_has_the_near_tie(orc, seed, delta_tols):
    SA, Sb, j0 = near_tie_problem(orc, seed, delta_tols=delta_tols)
    x, info = orc.nnls(SA, Sb)
    assert info["status"] == 0
    assert set(np.flatnonzero(x > 0)) == set(range(15)) | {j0}
    assert 0 < x[j0] < 1e-6 * np.max(x)


@pytest.mark.gpu
def test_accurate_mode_is_entered_and_matches_the_oracle(orc):
    import paper_0812_4547_gb300 as P

    ctx = P.Context(0)
    modes = []
    try:
        cases = ([dict(seed=s) for s in range(12)] + [dict(seed=100 + s, dependent=1e-3) for s in range(4)] +
                 [dict(seed=200 + s, delta_tols=5.0) for s in range(12)])
        for kw in cases:
            SA, Sb, j0 = near_tie_problem(orc, **kw)
            x_ref, info_ref = orc.nnls(SA, Sb)
            x, info = ctx.solve(dev_colmajor(SA), dev_vec(Sb))
            got = P.info_dict(info)
            xg = host(x)
            assert got["status"] == 0 and info_ref["status"] == 0
            assert np.array_equal(xg > 0, x_ref > 0), kw
            assert np.max(np.abs(xg - x_ref)) <= 1e-6 * np.max(np.abs(x_ref)), kw
            assert got["accurate_mode"] in (0, 1, 2) and got["reserved"] == 0
            modes.append(got["accurate_mode"])
    finally:
        ctx.close()
    # the FP32 iterations miss the near-tie in some of the problems
    assert sum(m > 0 for m in modes) >= 1, modes


@pytest.mark.gpu
def test_accurate_mode_in_batched_solves(orc):
    """The same problems through rnnls_solve_batched (one Lawson-Hanson block
    and one info per problem)."""
    import torch

    import paper_0812_4547_gb300 as P

    probs = [near_tie_problem(orc, seed) for seed in range(8)]
    probs += [near_tie_problem(orc, 200 + s, delta_tols=5.0) for s in range(8)]
    ctx = P.Context(0)
    try:
        tens = []
        for SA, Sb, _ in probs:
            tens.append((dev_colmajor(SA), dev_vec(Sb), torch.empty(SA.shape[1], dtype=torch.float64, device="cuda"),
                         torch.zeros(P.INFO_BYTES, dtype=torch.uint8, device="cuda")))
        ctx.solve_batched(tens)
        torch.cuda.synchronize()
        modes = []
        for (SA, Sb, _), (_, _, x, info) in zip(probs, tens):
            x_ref, _ = orc.nnls(SA, Sb)
            xg = host(x)
            assert np.array_equal(xg > 0, x_ref > 0)
            assert np.max(np.abs(xg - x_ref)) <= 1e-6 * np.max(np.abs(x_ref))
            modes.append(P.info_dict(info)["accurate_mode"])
        assert sum(m > 0 for m in modes) >= 1, modes
    finally:
        ctx.close()
