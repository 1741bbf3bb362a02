"""Seeded synthetic workloads shaped like the paper's NNLS problems.

This module only draws input data.  It holds none of the method's
arithmetic (no signs, no sampling, no transform, no solver), so both the
CUDA path and the FP64 oracle can be fed the same bytes from here.

The paper evaluates on TechTC300 term-document matrices (Sec. 4.1:
150-400 documents x 15k-35k terms, sparse and nonnegative) and on random
matrices of varying density (Sec. 4.2).  That dataset is not available, so
these generators stand in for it with the same shape class: tall, sparse,
nonnegative, heavy-tailed columns.

Recipe per column j (0-based) of a "term-document" matrix:
    entry = Bernoulli(density) * LogNormal(0, 1) * (j + 1) ** -zipf
with density 0.02 and zipf 1.1 by default (about 27 % of the rows of a
64-column matrix are entirely zero).  Targets are b = A x_true + eta with
x_true having an exact number of zeros at seeded random positions and
nonzeros uniform on [0, 2], and eta ~ N(0, sigma^2 I),
sigma = noise_rel * ||A x_true|| / sqrt(n).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

#: The five benchmark workloads.  Sizes are the full sizes; tests use
#: smaller n with the same recipe.
CONFIGS = {
    1: dict(name="plain-fp64 4096x20 uniform r=512", n=4096, d=20, r=512, dist="uniform", dtype="f64",
            zeros=10, noise_abs=0.01, seed=0),
    2: dict(name="plain-fp32 2^20x64 term-doc r=4096", n=2 ** 20, d=64, r=4096, dist="termdoc", dtype="f32",
            zero_frac=0.5, noise_rel=0.05, seed=2),
    3: dict(name="fp32 2^22x128 term-doc r=8192", n=2 ** 22, d=128, r=8192, dist="termdoc", dtype="f32",
            zero_frac=0.5, noise_rel=0.05, seed=3),
    4: dict(name="multi-rhs 2^20x100 + 256 rhs r=4096", n=2 ** 20, d=100, nrhs=256, r=4096, dist="termdoc",
            dtype="f32", zero_frac_range=(0.3, 0.8), noise_rel=0.05, seed=4),
    5: dict(name="uneven batch of 512", instances=512, n_log2_range=(14.0, 20.0), d_range=(16, 200),
            dist="termdoc", dtype="f32", zero_frac=0.5, noise_rel=0.05, seed=5),
}


@dataclass
class Problem:
    """One NNLS instance: A (n x d, column-major), b (n), the planted x_true."""
    A: np.ndarray
    b: np.ndarray
    x_true: np.ndarray
    r: int
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.A.shape[0]

    @property
    def d(self) -> int:
        return self.A.shape[1]


def termdoc_matrix(n: int, cols: int, rng: np.random.Generator, density: float = 0.02, zipf: float = 1.1,
                   col_offset: int = 0, dtype=np.float32) -> np.ndarray:
    """Sparse nonnegative heavy-tailed matrix stored dense, column-major."""
    A = np.zeros((n, cols), dtype=dtype, order="F")
    for j in range(cols):
        mask = rng.random(n, dtype=np.float32) < density
        k = int(mask.sum())
        vals = rng.lognormal(0.0, 1.0, k) * (j + col_offset + 1) ** (-zipf)
        A[mask, j] = vals.astype(dtype)
    return A


def planted_x(d: int, n_zero: int, rng: np.random.Generator) -> np.ndarray:
    """x_true with exactly n_zero zeros at seeded positions, the rest U[0, 2]."""
    x = rng.uniform(0.0, 2.0, d)
    x[rng.permutation(d)[:n_zero]] = 0.0
    return x


def _matvec64(A: np.ndarray, x: np.ndarray) -> np.ndarray:
    """A @ x accumulated in float64, one column at a time (no big temporaries)."""
    out = np.zeros(A.shape[0], dtype=np.float64)
    for j in range(A.shape[1]):
        if x[j] != 0.0:
            out += A[:, j].astype(np.float64) * x[j]
    return out


def noisy_target(A: np.ndarray, x: np.ndarray, rng: np.random.Generator, noise_rel: float | None = None,
                 noise_abs: float | None = None) -> np.ndarray:
    clean = _matvec64(A, x)
    n = A.shape[0]
    if noise_abs is not None:
        sigma = noise_abs
    else:
        sigma = noise_rel * float(np.linalg.norm(clean)) / math.sqrt(n)
    return clean + sigma * rng.standard_normal(n)


def next_pow2(v: float) -> int:
    p = 1
    while p < v:
        p <<= 1
    return p


def problem(config: int, n: int | None = None, d: int | None = None, r: int | None = None,
            seed: int | None = None) -> Problem:
    """Instance of workload ``config`` (1-4); n, d, r override the full sizes."""
    c = CONFIGS[config]
    n = c["n"] if n is None else n
    d = c["d"] if d is None else d
    r = c["r"] if r is None else r
    seed = c["seed"] if seed is None else seed
    rng = np.random.default_rng(seed)
    if c["dist"] == "uniform":
        A = np.asfortranarray(rng.random((n, d)))
        x = planted_x(d, min(c["zeros"], d), rng)
        b = noisy_target(A, x, rng, noise_abs=c["noise_abs"])
        return Problem(A=A, b=b, x_true=x, r=r, seed=seed, meta=dict(config=config, dtype="f64"))
    A = termdoc_matrix(n, d, rng)
    x = planted_x(d, int(round(c.get("zero_frac", 0.5) * d)), rng)
    b = noisy_target(A, x, rng, noise_rel=c["noise_rel"]).astype(np.float32)
    return Problem(A=A, b=b, x_true=x, r=r, seed=seed, meta=dict(config=config, dtype="f32"))


def multi_rhs(n: int | None = None, d: int | None = None, nrhs: int | None = None, r: int | None = None,
              seed: int | None = None):
    """Workload 4: shared A (n x d) and B (n x nrhs) of NMF-style targets.

    Target j is A x_j + noise, x_j with round(f_j d) zeros, f_j ~ U[0.3, 0.8]."""
    c = CONFIGS[4]
    n = c["n"] if n is None else n
    d = c["d"] if d is None else d
    nrhs = c["nrhs"] if nrhs is None else nrhs
    r = c["r"] if r is None else r
    seed = c["seed"] if seed is None else seed
    rng = np.random.default_rng(seed)
    A = termdoc_matrix(n, d, rng)
    lo, hi = c["zero_frac_range"]
    X = np.zeros((d, nrhs))
    B = np.zeros((n, nrhs), dtype=np.float32, order="F")
    for j in range(nrhs):
        f = rng.uniform(lo, hi)
        X[:, j] = planted_x(d, int(round(f * d)), rng)
        B[:, j] = noisy_target(A, X[:, j], rng, noise_rel=c["noise_rel"]).astype(np.float32)
    return A, B, X, r


def batch_shapes(count: int | None = None, seed: int | None = None, n_log2_range=None, d_range=None):
    """Workload 5 shapes: list of (n_raw, d, r).

    n_raw = floor(2^U[14, 20]), d ~ U{16..200}, r = next pow2 of 8 (d+1) ln n
    with n the padded size."""
    c = CONFIGS[5]
    count = c["instances"] if count is None else count
    seed = c["seed"] if seed is None else seed
    lo, hi = c["n_log2_range"] if n_log2_range is None else n_log2_range
    dlo, dhi = c["d_range"] if d_range is None else d_range
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n_raw = int(math.floor(2.0 ** rng.uniform(lo, hi)))
        d = int(rng.integers(dlo, dhi + 1))
        n_pad = next_pow2(n_raw)
        r = next_pow2(8.0 * (d + 1) * math.log(n_pad))
        out.append((n_raw, d, r))
    return out


def batch_instance(i: int, n_raw: int, d: int, r: int, seed: int | None = None) -> Problem:
    """Data of instance i of workload 5 (same recipe as workload 2)."""
    c = CONFIGS[5]
    base = c["seed"] if seed is None else seed
    rng = np.random.default_rng([base, i])
    A = termdoc_matrix(n_raw, d, rng)
    x = planted_x(d, int(round(c["zero_frac"] * d)), rng)
    b = noisy_target(A, x, rng, noise_rel=c["noise_rel"]).astype(np.float32)
    return Problem(A=A, b=b, x_true=x, r=r, seed=base, meta=dict(config=5, instance=i, dtype="f32"))
