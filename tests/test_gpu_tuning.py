"""The launch-shape knobs (rnnls_tuning) and the autotuner on the GPU: a
tuned plan must give the same sketch (rows bit-exact, values to FP32
summation order) and the same solve as the default plan."""
import numpy as np
import pytest

from tests.gpu_util import dev_colmajor, dev_vec, host, rel_fro

pytestmark = pytest.mark.gpu


def test_tuning_round_trip_and_validation():
    import paper_0812_4547_gb300 as P
    from paper_0812_4547_gb300 import _binding as B

    ctx = P.Context(0)
    try:
        assert all(v == 0 for v in ctx.get_tuning().values())
        t = {"sketch_sms": 100, "full_step_min_slots": 64, "gram_min_chunks": 4, "gram_max_splits": 16,
             "batch_gram_chunks": 64, "batch_step_cost": 200, "lh_warp_max_d": 96}
        ctx.set_tuning(t)
        assert ctx.get_tuning() == t
        for bad in ({"full_step_min_slots": 47}, {"gram_max_splits": 1025}, {"sketch_sms": -1},
                    {"batch_step_cost": 100001}, {"lh_warp_max_d": -1}, {"lh_warp_max_d": 1025}):
            with pytest.raises(B.RNNLSError) as e:
                ctx.set_tuning(bad)
            assert e.value.status == B.RNNLS_EINVAL
        assert ctx.get_tuning() == t  # a refused setting changes nothing
        ctx.set_sketch_sms(7)
        assert ctx.get_tuning()["sketch_sms"] == 7
    finally:
        ctx.close()


def _sketch(ctx, A, b, r, seed):
    SA, Sb, idx, _ = ctx.sketch(A, b, r, seed=seed)
    return host(SA), host(Sb), host(idx)


def test_full_step_threshold_gives_the_same_sketch():
    """r = 16384 has 64 rows per thread: by default the step's chunks are
    combined by H_4 first; with the threshold above 64 they are not."""
    import paper_0812_4547_gb300 as P

    rng = np.random.default_rng(1)
    n, d, r = (1 << 18) + 11, 5, 16384
    A = dev_colmajor(rng.standard_normal((n, d)), np.float32)
    b = dev_vec(rng.standard_normal(n), np.float32)
    ctx = P.Context(0)
    try:
        SA0, Sb0, i0 = _sketch(ctx, A, b, r, 3)
        ctx.set_tuning({"full_step_min_slots": 1024})
        SA1, Sb1, i1 = _sketch(ctx, A, b, r, 3)
        ctx.set_tuning({"full_step_min_slots": 64})
        SA2, Sb2, i2 = _sketch(ctx, A, b, r, 3)
    finally:
        ctx.close()
    assert np.array_equal(i0, i1) and np.array_equal(i0, i2)
    for SA, Sb in ((SA1, Sb1), (SA2, Sb2)):
        assert rel_fro(SA, SA0.astype(np.float64)) <= 1e-6 and rel_fro(Sb, Sb0.astype(np.float64)) <= 1e-6


def test_gram_split_knobs_give_the_same_gram_and_solve():
    import paper_0812_4547_gb300 as P

    rng = np.random.default_rng(2)
    r, d = 8192, 100
    SA = dev_colmajor(rng.standard_normal((r, d)) * np.exp(rng.standard_normal(d)), np.float32)
    Sb = dev_vec(rng.standard_normal(r), np.float32)
    ctx = P.Context(0)
    try:
        Q0, _ = ctx.gram(SA, Sb)
        x0, _ = ctx.solve(SA, Sb)
        Q0, x0 = host(Q0), host(x0)
        for t in ({"gram_min_chunks": 1, "gram_max_splits": 64}, {"gram_min_chunks": 32, "gram_max_splits": 1}):
            ctx.set_tuning(t)
            Q1, _ = ctx.gram(SA, Sb)
            x1, _ = ctx.solve(SA, Sb)
            Q1, x1 = host(Q1), host(x1)
            diag = np.sqrt(np.diag(Q0))
            assert np.max(np.abs(Q1 - Q0) / np.outer(diag, diag)) <= 1e-13, t
            assert np.array_equal(x1 > 0, x0 > 0)
            assert np.max(np.abs(x1 - x0)) <= 1e-6 * np.max(np.abs(x0))
    finally:
        ctx.close()


def test_batched_knobs_give_the_same_batch():
    import torch

    import paper_0812_4547_gb300 as P

    rng = np.random.default_rng(4)
    shapes = [(40000, 30, 8192), (20000, 120, 16384), (70000, 9, 4096)]
    inst = [(dev_colmajor(rng.standard_normal((n, d)), np.float32), dev_vec(rng.standard_normal(n), np.float32), r)
            for n, d, r in shapes]

    def run(ctx):
        outs = []
        for (A, b, r) in inst:
            d = A.shape[1]
            outs.append((torch.empty((d, r), device="cuda").t(), torch.empty(r, device="cuda"),
                         torch.empty(r, dtype=torch.int32, device="cuda"),
                         torch.empty(d, dtype=torch.float64, device="cuda")))
        ctx.sketch_batched([(A, b, r, 5 + i, 0, o[0], o[1], o[2]) for i, ((A, b, r), o) in enumerate(zip(inst, outs))])
        ctx.solve_batched([(o[0], o[1], o[3], None) for o in outs])
        torch.cuda.synchronize()
        return [tuple(host(t) for t in o) for o in outs]

    ctx = P.Context(0)
    try:
        ref = run(ctx)
        ctx.set_tuning({"batch_gram_chunks": 32, "batch_step_cost": 300, "full_step_min_slots": 1024})
        got = run(ctx)
    finally:
        ctx.close()
    for (SA0, Sb0, i0, x0), (SA1, Sb1, i1, x1) in zip(ref, got):
        assert np.array_equal(i0, i1)
        assert rel_fro(SA1, SA0.astype(np.float64)) <= 1e-6 and rel_fro(Sb1, Sb0.astype(np.float64)) <= 1e-6
        assert np.max(np.abs(x1 - x0)) <= 1e-6 * np.max(np.abs(x0))


def test_autotuner_end_to_end(tmp_path):
    import paper_0812_4547_gb300 as P
    from paper_0812_4547_gb300 import autotune as T

    rng = np.random.default_rng(6)
    n, d, r = 1 << 17, 40, 4096
    A = dev_colmajor(rng.standard_normal((n, d)), np.float32)
    b = dev_vec(rng.standard_normal(n), np.float32)
    ctx = P.Context(0)
    path = str(tmp_path / "tuning.json")
    cands = {"full_step_min_slots": [0, 1024], "gram_min_chunks": [0, 32], "gram_max_splits": [0, 4]}
    try:
        def step():
            SA, Sb, _, _ = ctx.sketch(A, b, r, seed=1, want_count=False)
            ctx.solve(SA, Sb)

        e1 = T.tune(ctx, step, "single", {"n": n, "d": d, "r": r}, path=path, repeats=2, candidates=cands)
        assert not e1["cached"] and len(e1["trials"]) == 4
        assert e1["ms"] <= e1["default_ms"]
        assert ctx.get_tuning() == {**ctx.get_tuning(), **e1["tuning"]}
        e2 = T.tune(ctx, step, "single", {"n": n, "d": d, "r": r}, path=path, candidates=cands)
        assert e2["cached"] and e2["tuning"] == e1["tuning"]
        assert e1["key"] in T.load_cache(path)["entries"]
    finally:
        ctx.close()


@pytest.mark.parametrize("d", [8, 40, 64, 100])
def test_lh_team_size_gives_the_same_solve(orc, d):
    """Lawson-Hanson as one-warp blocks or as 256-thread blocks: the same
    active set and x within 1e-6 of the oracle's (one problem and a batch)."""
    import torch

    import paper_0812_4547_gb300 as P

    rng = np.random.default_rng(d)
    r = 2048
    SAh = (rng.standard_normal((r, d)) * np.exp(rng.standard_normal(d))).astype(np.float32)
    x0 = np.abs(rng.standard_normal(d)) * (rng.random(d) < 0.5)
    Sbh = (SAh.astype(np.float64) @ x0 + rng.standard_normal(r)).astype(np.float32)
    x_ref, _ = orc.nnls(SAh, Sbh)
    SA, Sb = dev_colmajor(SAh), dev_vec(Sbh)
    ctx = P.Context(0)
    try:
        for wmd in (0, 64, 1024):
            ctx.set_tuning({"lh_warp_max_d": wmd})
            x, info = ctx.solve(SA, Sb)
            xs = torch.empty(d, dtype=torch.float64, device="cuda")
            infos = torch.zeros(P.INFO_BYTES, dtype=torch.uint8, device="cuda")
            ctx.solve_batched([(SA, Sb, xs, infos)])
            torch.cuda.synchronize()
            for xg, inf in ((host(x), info), (host(xs), infos)):
                assert P.info_dict(inf)["status"] == 0
                assert np.array_equal(xg > 0, x_ref > 0), wmd
                assert np.max(np.abs(xg - x_ref)) <= 1e-6 * np.max(np.abs(x_ref)), wmd
    finally:
        ctx.close()
