"""FP64 CPU oracle for RandomizedNNLS (Boutsidis & Drineas).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py`` may import this
package.  The CUDA library never loads it and shares no code with it.

The arithmetic lives in ``rnnls_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off`` so that both x86-64 and AArch64 hosts round alike);
this module compiles it with gcc and exposes numpy-level wrappers:

* :func:`philox4x64_10`, :func:`signs`, :func:`sample` -- the randomness of
  Alg. 1 steps 2-4 (generator: Salmon et al., SC'11).
* :func:`hadamard_dense`, :func:`fwht` -- the Sylvester matrix of Sec. 2.
* :func:`sketch`, :func:`sketch_entry` -- H~ D [A b] of Alg. 1.
* :func:`gram`, :func:`nnls_lh`, :func:`nnls`, :func:`lh_tol` -- the
  Lawson-Hanson solve of Alg. 1 step 5 on the QP form of Sec. 3.4.
* :func:`residual_sq`, :func:`randomized_nnls`, :func:`exact_nnls` --
  Definition 1's objective and the residual ratio of Theorem 1.
* :func:`boosted_nnls` -- repetitions of Alg. 1, best full residual kept
  (the footnote to Theorem 1).
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rnnls_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = None
_LOCK = threading.Lock()

MODE_IID = 0
MODE_BERNOULLI = 1

OK = 0
EINVAL = 1
ECAPACITY = 2
ESINGULAR = 4
EMAXITER = 5


def _lib_path() -> str:
    return os.path.join(_BUILD, f"liboracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (gcc, FP64, OpenMP if present)."""
    out = _lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    tmp = out + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, out)
    return out


class _LHInfo(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("outer_iters", ctypes.c_int32),
        ("inner_iters", ctypes.c_int32),
        ("passive_count", ctypes.c_int32),
        ("trace_len", ctypes.c_int64),
    ]


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            U64 = ctypes.c_uint64
            D = ctypes.c_double
            lib.orc_philox4x64_10.argtypes = [P, P, P]
            lib.orc_philox4x64_10.restype = None
            lib.orc_sign.argtypes = [U64, U64, U64]
            lib.orc_sign.restype = ctypes.c_int
            lib.orc_signs.argtypes = [U64, U64, I64, P]
            lib.orc_signs.restype = None
            lib.orc_sample.argtypes = [U64, U64, I64, I64, ctypes.c_int, P, I64]
            lib.orc_sample.restype = I64
            lib.orc_scale.argtypes = [I64, I64, ctypes.c_int]
            lib.orc_scale.restype = D
            lib.orc_hadamard_dense.argtypes = [I64, P]
            lib.orc_hadamard_dense.restype = None
            lib.orc_fwht.argtypes = [P, I64]
            lib.orc_fwht.restype = None
            lib.orc_sketch.argtypes = [P, I64, P, I64, I64, I64, U64, U64, ctypes.c_int, P, I64, P, P, I64,
                                       ctypes.c_int]
            lib.orc_sketch.restype = I64
            lib.orc_sketch_entry.argtypes = [P, I64, U64, U64, I64, D]
            lib.orc_sketch_entry.restype = D
            lib.orc_gram.argtypes = [P, I64, P, I64, I64, P, P, P]
            lib.orc_gram.restype = None
            lib.orc_lh_tol.argtypes = [P, I64, P, I64, I64]
            lib.orc_lh_tol.restype = D
            lib.orc_nnls_lh.argtypes = [P, P, I64, D, I64, I64, P, ctypes.POINTER(_LHInfo)]
            lib.orc_nnls_lh.restype = ctypes.c_int
            lib.orc_nnls_lh_traced.argtypes = [P, P, I64, D, I64, I64, P, ctypes.POINTER(_LHInfo), P, I64]
            lib.orc_nnls_lh_traced.restype = ctypes.c_int
            lib.orc_nnls.argtypes = [P, I64, P, I64, I64, P, ctypes.POINTER(_LHInfo)]
            lib.orc_nnls.restype = ctypes.c_int
            lib.orc_residual_sq.argtypes = [P, I64, P, I64, I64, P]
            lib.orc_residual_sq.restype = D
            lib.orc_max_threads.argtypes = []
            lib.orc_max_threads.restype = ctypes.c_int
            _LIB = lib
    return _LIB


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _f64_colmajor(A) -> np.ndarray:
    return np.asfortranarray(np.asarray(A, dtype=np.float64))


def max_threads() -> int:
    return int(_lib().orc_max_threads())


# --------------------------------------------------------------------------
# randomness
# --------------------------------------------------------------------------
def philox4x64_10(ctr, key) -> np.ndarray:
    """One Philox4x64-10 block: 4 uint64 words for counter ``ctr`` (4 words), key ``key`` (2 words)."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint64))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64))
    out = np.zeros(4, dtype=np.uint64)
    _lib().orc_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def signs(seed: int, instance: int, n: int) -> np.ndarray:
    """Diagonal of D (Alg. 1 step 4) for rows 0..n-1, as int8 +-1."""
    D = np.zeros(n, dtype=np.int8)
    _lib().orc_signs(seed, instance, n, _ptr(D))
    return D


def padded_n(n_raw: int) -> int:
    n = 1
    while n < n_raw:
        n <<= 1
    return n


def bernoulli_capacity(r: int) -> int:
    """Rows an output must be able to hold in Bernoulli mode (about 6 sigma above r)."""
    import math
    return int(r + math.ceil(6.0 * math.sqrt(r)) + 16)


def sample(seed: int, instance: int, n: int, r: int, mode: int = MODE_IID, cap: int | None = None) -> np.ndarray:
    """Sampled row indices of H~ (Alg. 1 steps 2-3); n must be the padded size."""
    if cap is None:
        cap = r if mode == MODE_IID else max(n if r >= n else bernoulli_capacity(r), 1)
    idx = np.zeros(max(cap, 1), dtype=np.int32)
    cnt = _lib().orc_sample(seed, instance, n, r, mode, _ptr(idx), cap)
    if cnt < 0:
        raise ValueError("sample capacity exceeded")
    return idx[:cnt].copy()


def scale(n: int, r: int, mode: int = MODE_IID) -> float:
    return float(_lib().orc_scale(n, r, mode))


# --------------------------------------------------------------------------
# Hadamard
# --------------------------------------------------------------------------
def hadamard_dense(n: int) -> np.ndarray:
    """Unnormalised Sylvester matrix H_n (Sec. 2), natural order."""
    H = np.zeros((n, n), dtype=np.float64)
    _lib().orc_hadamard_dense(n, _ptr(H))
    return H


def fwht(y) -> np.ndarray:
    """Unnormalised fast transform H_n y (iterative butterflies)."""
    v = np.ascontiguousarray(np.asarray(y, dtype=np.float64)).copy()
    _lib().orc_fwht(_ptr(v), v.shape[0])
    return v


# --------------------------------------------------------------------------
# sketch
# --------------------------------------------------------------------------
def sketch(A, b, r: int, seed: int, instance: int = 0, mode: int = MODE_IID, nthreads: int = 1):
    """SA, Sb, idx of Alg. 1 for A (n_raw x d) and b (n_raw), FP64.

    Inputs are promoted to FP64 exactly (FP32 inputs keep their bytes)."""
    A64 = _f64_colmajor(A)
    b64 = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
    n_raw, d = A64.shape
    n = padded_n(n_raw)
    cap = r if mode == MODE_IID else (n if r >= n else bernoulli_capacity(r))
    SA = np.zeros((cap, d), dtype=np.float64, order="F")
    Sb = np.zeros(cap, dtype=np.float64)
    idx = np.zeros(cap, dtype=np.int32)
    rr = _lib().orc_sketch(_ptr(A64), n_raw, _ptr(b64), n_raw, d, r, seed, instance, mode, _ptr(SA), cap,
                           _ptr(Sb), _ptr(idx), cap, nthreads)
    if rr < 0:
        raise ValueError(f"oracle sketch failed: {-rr}")
    return np.asfortranarray(SA[:rr]), Sb[:rr].copy(), idx[:rr].copy()


def sketch_entry(x, seed: int, instance: int, row: int, scale_: float) -> float:
    """One sketch entry from the definition, O(n): scale * sum_i H[row, i] D_i x_i."""
    v = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    return float(_lib().orc_sketch_entry(_ptr(v), v.shape[0], seed, instance, row, scale_))


# --------------------------------------------------------------------------
# NNLS
# --------------------------------------------------------------------------
def gram(S, s):
    S64 = _f64_colmajor(S)
    s64 = np.ascontiguousarray(np.asarray(s, dtype=np.float64))
    m, d = S64.shape
    Q = np.zeros((d, d), dtype=np.float64)
    q = np.zeros(d, dtype=np.float64)
    ss = np.zeros(1, dtype=np.float64)
    _lib().orc_gram(_ptr(S64), max(m, 1), _ptr(s64), m, d, _ptr(Q), _ptr(q), _ptr(ss))
    return Q, q, float(ss[0])


def lh_tol(S, s) -> float:
    S64 = _f64_colmajor(S)
    s64 = np.ascontiguousarray(np.asarray(s, dtype=np.float64))
    m, d = S64.shape
    return float(_lib().orc_lh_tol(_ptr(S64), max(m, 1), _ptr(s64), m, d))


def nnls_lh(Q, q, tol: float, max_outer: int | None = None, max_inner: int | None = None, trace: bool = False):
    """Lawson-Hanson on the QP form; returns (x, info dict).

    With ``trace=True`` the info dict also holds ``trace``: the objective
    x'Qx/2 - q'x after every update of x."""
    Q64 = np.ascontiguousarray(np.asarray(Q, dtype=np.float64))
    q64 = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
    d = q64.shape[0]
    x = np.zeros(d, dtype=np.float64)
    info = _LHInfo()
    mo = 3 * d if max_outer is None else max_outer
    mi = 30 * d if max_inner is None else max_inner
    cap = 4 * (mo + mi) + 8
    tr = np.zeros(cap, dtype=np.float64)
    _lib().orc_nnls_lh_traced(_ptr(Q64), _ptr(q64), d, tol, mo, mi, _ptr(x), ctypes.byref(info), _ptr(tr), cap)
    out = _info_dict(info)
    if trace:
        out["trace"] = tr[:min(info.trace_len, cap)].copy()
    return x, out


def _info_dict(info: _LHInfo) -> dict:
    return {"status": info.status, "outer_iters": info.outer_iters, "inner_iters": info.inner_iters,
            "passive_count": info.passive_count}


def nnls(S, s):
    """argmin_{x>=0} ||S x - s||^2 by Lawson-Hanson with the default tolerance and caps."""
    S64 = _f64_colmajor(S)
    s64 = np.ascontiguousarray(np.asarray(s, dtype=np.float64))
    m, d = S64.shape
    x = np.zeros(d, dtype=np.float64)
    info = _LHInfo()
    _lib().orc_nnls(_ptr(S64), max(m, 1), _ptr(s64), m, d, _ptr(x), ctypes.byref(info))
    return x, _info_dict(info)


def residual_sq(A, b, x) -> float:
    """||A x - b||^2 in FP64 (Definition 1)."""
    A64 = _f64_colmajor(A)
    b64 = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
    x64 = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    n, d = A64.shape
    return float(_lib().orc_residual_sq(_ptr(A64), max(n, 1), _ptr(b64), n, d, _ptr(x64)))


def randomized_nnls(A, b, r: int, seed: int, instance: int = 0, mode: int = MODE_IID, nthreads: int = 1):
    """Alg. 1 end to end: sketch, then Lawson-Hanson on the sketch."""
    SA, Sb, idx = sketch(A, b, r, seed, instance, mode, nthreads)
    x, info = nnls(SA, Sb)
    return x, info, (SA, Sb, idx)


def boosted_nnls(A, b, r: int, seed: int, k: int, instance0: int = 0, mode: int = MODE_IID, nthreads: int = 1):
    """Repeated RandomizedNNLS (the footnote to Theorem 1 in Sec. 1: a few
    independent repetitions raise the success probability of the (1 + eps)
    bound).  Repetition j runs Alg. 1 with randomness (seed, instance0 + j);
    the answer is the repetition with the smallest full residual
    ||A x_j - b||^2 among those whose Lawson-Hanson solve ended with status
    OK (ties to the smallest j; if none did, repetition 0).

    Returns (x, best, residuals, infos): residuals[j] = ||A x_j - b||^2 for
    every repetition, infos[j] its solve's info."""
    if k < 1:
        raise ValueError("k >= 1 repetitions")
    xs, res, infos = [], [], []
    for j in range(k):
        x, info, _ = randomized_nnls(A, b, r, seed, instance0 + j, mode, nthreads)
        xs.append(x)
        infos.append(info)
        res.append(residual_sq(A, b, x))
    best = -1
    for j in range(k):
        if infos[j]["status"] == OK and np.isfinite(res[j]) and (best < 0 or res[j] < res[best]):
            best = j
    best = max(best, 0)
    return xs[best], best, np.array(res, dtype=np.float64), infos


def exact_nnls(A, b):
    """x_opt of Definition 1 on the full A (Lawson-Hanson on A'A, A'b)."""
    return nnls(A, b)
