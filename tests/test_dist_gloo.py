"""Multi-process paths on CPU (gloo, world sizes 2 and 4).

1. The row-shard identity behind rnnls_sketch_shard: with the rows split
   into G blocks, rank g transforms only its block with the length-n/G
   Hadamard matrix, keeps the sampled rows i mod (n/G) with the sign
   (-1)^popcount((i div n/G) & g), and one sum-reduce gives the full sketch
   (H_n = H_G (x) H_{n/G}, Sec. 2's Sylvester recursion).  Every piece here
   is the FP64 oracle's; the reduce is gloo's.
2. bench.py's multi-rank bookkeeping: distinct instances per rank and the
   slowest rank's time.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank: int, world: int, port: int):
    import sys

    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _shard_worker(rank: int, world: int, port: int, n_raw: int, d: int, r: int, out_dir: str):
    _init(rank, world, port)
    import oracle

    oracle.build()
    rng = np.random.default_rng(7)
    A = rng.standard_normal((n_raw, d))
    b = rng.standard_normal(n_raw)
    seed, inst = 4, 1
    n = oracle.padded_n(n_raw)
    m = n // world
    X = np.zeros((n, d + 1))
    X[:n_raw, :d] = A
    X[:n_raw, d] = b
    D = oracle.signs(seed, inst, n).astype(np.float64)
    idx = oracle.sample(seed, inst, n, r)
    s = oracle.scale(n, r)
    rows = slice(rank * m, (rank + 1) * m)
    P = np.zeros((r, d + 1))
    for col in range(d + 1):
        z = oracle.fwht(D[rows] * X[rows, col])
        for k, i in enumerate(idx):
            sign = -1.0 if bin((int(i) // m) & rank).count("1") % 2 else 1.0
            P[k, col] = s * sign * z[int(i) % m]
    t = torch.from_numpy(P)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    if rank == 0:
        SA, Sb, idx_o = oracle.sketch(A, b, r, seed, inst)
        np.save(os.path.join(out_dir, "sum.npy"), t.numpy())
        np.save(os.path.join(out_dir, "full.npy"), np.column_stack([SA, Sb]))
    dist.destroy_process_group()


@pytest.mark.parametrize("n_raw,d,r,world", [(3000, 3, 200, 2), (1 << 12, 2, 5000, 2), (3000, 3, 200, 4),
                                            ((1 << 13) + 5, 2, 700, 4)])
def test_row_shard_sum_reduce_gives_the_sketch(tmp_path, n_raw, d, r, world):
    mp.spawn(_shard_worker, args=(world, _free_port(), n_raw, d, r, str(tmp_path)), nprocs=world, join=True)
    got = np.load(tmp_path / "sum.npy")
    want = np.load(tmp_path / "full.npy")
    assert np.max(np.abs(got - want)) <= 1e-12 * max(1.0, np.max(np.abs(want)))


def _bench_worker(rank: int, world: int, port: int, out_dir: str):
    _init(rank, world, port)
    import bench

    os.environ["WORLD_SIZE"] = str(world)
    os.environ["RANK"] = str(rank)
    ws, rk, _ = bench.dist_env()
    seed = bench.rank_seed(10, rk, ws)
    slowest = bench.max_over_ranks(1.5 + rank, torch.device("cpu"))
    seeds = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(seeds, torch.tensor([seed]))
    if rank == 0:
        np.save(os.path.join(out_dir, "bench.npy"), np.array([slowest] + [int(x) for x in seeds]))
    dist.destroy_process_group()


def test_bench_rank_bookkeeping(tmp_path):
    world = 2
    mp.spawn(_bench_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = np.load(tmp_path / "bench.npy")
    assert res[0] == 2.5  # the slower rank's time
    assert len(set(res[1:].tolist())) == world  # one instance per rank
