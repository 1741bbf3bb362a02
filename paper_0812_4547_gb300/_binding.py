"""ctypes declarations of the C ABI in include/rnnls.h (librnnls.so).

Argument marshalling only: every step of the method runs in the CUDA
library.  Importing this module never builds anything; :func:`lib` raises
if ``librnnls.so`` is missing, so no caller can fall back to another path.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

RNNLS_OK = 0
RNNLS_EINVAL = 1
RNNLS_ECAPACITY = 2
RNNLS_ENONFINITE = 3
RNNLS_ESINGULAR = 4
RNNLS_EMAXITER = 5
RNNLS_ETIMEOUT = 6
RNNLS_ECUDA = 7
RNNLS_ENOMEM = 8
RNNLS_EUNSUPPORTED = 9

RNNLS_SAMPLE_IID = 0
RNNLS_SAMPLE_BERNOULLI = 1
RNNLS_PREC_FP32 = 0
RNNLS_PREC_BF16X2 = 2

#: every entry point declared in include/rnnls.h
EXPORTS = (
    "rnnls_create", "rnnls_destroy", "rnnls_set_stream", "rnnls_sketch", "rnnls_sketch_f64", "rnnls_solve",
    "rnnls_solve_f64", "rnnls_solve_batched", "rnnls_residual", "rnnls_strerror", "rnnls_profile_begin",
    "rnnls_profile_end", "rnnls_sketch_noalloc", "rnnls_set_sketch_sms", "rnnls_sketch_multi", "rnnls_sketch_shard",
    "rnnls_solve_multi", "rnnls_sketch_batched", "rnnls_solve_boosted", "rnnls_set_plan_event", "rnnls_gram",
    "rnnls_solve_pg", "rnnls_sketch_csc", "rnnls_set_tuning", "rnnls_get_tuning",
    "rnnls_solve_batched_device", "rnnls_sketch_batched_ex",
)


class rnnls_info(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("outer_iters", ctypes.c_int32),
        ("inner_iters", ctypes.c_int32),
        ("passive_count", ctypes.c_int32),
        ("tol", ctypes.c_double),
        ("dual_max", ctypes.c_double),
        ("objective", ctypes.c_double),
        ("accurate_mode", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class rnnls_tuning(ctypes.Structure):
    _fields_ = [
        ("sketch_sms", ctypes.c_int32),
        ("full_step_min_slots", ctypes.c_int32),
        ("gram_min_chunks", ctypes.c_int32),
        ("gram_max_splits", ctypes.c_int32),
        ("batch_gram_chunks", ctypes.c_int32),
        ("batch_step_cost", ctypes.c_int32),
        ("lh_warp_max_d", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


#: the tuning knobs by name (rnnls_tuning's fields other than reserved)
TUNING_KNOBS = tuple(f[0] for f in rnnls_tuning._fields_ if f[0] != "reserved")


class rnnls_kernel_time(ctypes.Structure):
    _fields_ = [
        ("name", ctypes.c_char * 32),
        ("launches", ctypes.c_int64),
        ("total_ms", ctypes.c_double),
    ]


class rnnls_sketch_job(ctypes.Structure):
    _fields_ = [
        ("A", ctypes.c_void_p),
        ("lda", ctypes.c_int64),
        ("b", ctypes.c_void_p),
        ("n_raw", ctypes.c_int64),
        ("d", ctypes.c_int64),
        ("r", ctypes.c_int64),
        ("seed", ctypes.c_uint64),
        ("instance", ctypes.c_uint64),
        ("SA", ctypes.c_void_p),
        ("ldsa", ctypes.c_int64),
        ("Sb", ctypes.c_void_p),
        ("idx", ctypes.c_void_p),
    ]


class rnnls_problem(ctypes.Structure):
    _fields_ = [
        ("SA", ctypes.c_void_p),
        ("ldsa", ctypes.c_int64),
        ("Sb", ctypes.c_void_p),
        ("r", ctypes.c_int64),
        ("d", ctypes.c_int64),
        ("x", ctypes.c_void_p),
        ("info", ctypes.c_void_p),
    ]


_LIB = None
_LOCK = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """The loaded CUDA library (raises if it has not been built)."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(path)
        P, I64, U64, U32, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        L.rnnls_create.argtypes = [ctypes.POINTER(P), I32, P]
        L.rnnls_destroy.argtypes = [P]
        L.rnnls_set_stream.argtypes = [P, P]
        L.rnnls_set_sketch_sms.argtypes = [P, I32]
        L.rnnls_set_plan_event.argtypes = [P, P]
        sk = [P, P, I64, P, I64, I64, I64, U64, U64, U32, P, I64, P, P, I64, ctypes.POINTER(I64)]
        L.rnnls_sketch.argtypes = sk
        L.rnnls_sketch_f64.argtypes = sk
        L.rnnls_solve.argtypes = [P, P, I64, P, I64, I64, P, P]
        L.rnnls_solve_f64.argtypes = [P, P, I64, P, I64, I64, P, P]
        L.rnnls_solve_batched.argtypes = [P, ctypes.POINTER(rnnls_problem), I64, U32]
        L.rnnls_solve_multi.argtypes = [P, P, I64, P, I64, I64, I64, I64, P, I64, P]
        L.rnnls_gram.argtypes = [P, P, I64, P, I64, I64, P, P]
        L.rnnls_solve_pg.argtypes = [P, P, I64, P, I64, I64, P, P, ctypes.c_double, I32]
        L.rnnls_sketch_csc.argtypes = [P, P, P, P, P, I64, I64, I64, U64, U64, P, I64, P, P]
        L.rnnls_solve_batched_device.argtypes = [P, P, I64, I64, I64, U32]
        L.rnnls_set_tuning.argtypes = [P, ctypes.POINTER(rnnls_tuning)]
        L.rnnls_get_tuning.argtypes = [P, ctypes.POINTER(rnnls_tuning)]
        L.rnnls_sketch_batched.argtypes = [P, ctypes.POINTER(rnnls_sketch_job), I64]
        L.rnnls_sketch_batched_ex.argtypes = [P, ctypes.POINTER(rnnls_sketch_job), I64, U32]
        L.rnnls_residual.argtypes = [P, P, I64, P, I64, I64, P, P]
        L.rnnls_solve_boosted.argtypes = [P, P, I64, P, I64, I64, I64, U64, U64, I32, P, P, P, P]
        L.rnnls_profile_begin.argtypes = [P, I32]
        L.rnnls_profile_end.argtypes = [P, ctypes.POINTER(rnnls_kernel_time), I32, ctypes.POINTER(I32)]
        L.rnnls_sketch_noalloc.argtypes = [P, P, I64, P, I64, I64, I64, U64, U64, P, I64, P, P]
        L.rnnls_sketch_multi.argtypes = [P, P, I64, P, I64, I64, I64, I64, I64, U64, U64, P, I64, P, I64, P]
        L.rnnls_sketch_shard.argtypes = [P, P, I64, P, I64, I64, I64, I64, I64, U64, U64, P, I64, P, P]
        L.rnnls_strerror.argtypes = [I32]
        L.rnnls_strerror.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name != "rnnls_strerror":
                getattr(L, name).restype = I32
        _LIB = L
        return L


class RNNLSError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().rnnls_strerror(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")


def check(status: int, where: str) -> None:
    if status != RNNLS_OK:
        raise RNNLSError(status, where)


# thin same-name wrappers over raw pointers -------------------------------------------------

def rnnls_create(device: int = 0, stream: int = 0) -> int:
    h = ctypes.c_void_p()
    check(lib().rnnls_create(ctypes.byref(h), device, ctypes.c_void_p(stream)), "rnnls_create")
    return h.value


def rnnls_destroy(ctx: int) -> None:
    check(lib().rnnls_destroy(ctypes.c_void_p(ctx)), "rnnls_destroy")


def rnnls_set_stream(ctx: int, stream: int) -> None:
    check(lib().rnnls_set_stream(ctypes.c_void_p(ctx), ctypes.c_void_p(stream)), "rnnls_set_stream")


def rnnls_set_sketch_sms(ctx: int, sms: int) -> None:
    check(lib().rnnls_set_sketch_sms(ctypes.c_void_p(ctx), sms), "rnnls_set_sketch_sms")


def rnnls_set_plan_event(ctx: int, event: int) -> None:
    check(lib().rnnls_set_plan_event(ctypes.c_void_p(ctx), ctypes.c_void_p(event)), "rnnls_set_plan_event")


def _sketch(fn, name, ctx, A, lda, b, n_raw, d, r, seed, instance, flags, SA, ldsa, Sb, idx, cap, want_count):
    rout = ctypes.c_int64(-1)
    st = fn(ctypes.c_void_p(ctx), ctypes.c_void_p(A), lda, ctypes.c_void_p(b), n_raw, d, r, seed, instance, flags,
            ctypes.c_void_p(SA), ldsa, ctypes.c_void_p(Sb), ctypes.c_void_p(idx), cap,
            ctypes.byref(rout) if want_count else None)
    check(st, name)
    return rout.value


def rnnls_sketch(ctx, A, lda, b, n_raw, d, r, seed, instance, flags, SA, ldsa, Sb, idx, cap, want_count=True):
    return _sketch(lib().rnnls_sketch, "rnnls_sketch", ctx, A, lda, b, n_raw, d, r, seed, instance, flags, SA, ldsa,
                   Sb, idx, cap, want_count)


def rnnls_sketch_f64(ctx, A, lda, b, n_raw, d, r, seed, instance, flags, SA, ldsa, Sb, idx, cap, want_count=True):
    return _sketch(lib().rnnls_sketch_f64, "rnnls_sketch_f64", ctx, A, lda, b, n_raw, d, r, seed, instance, flags, SA,
                   ldsa, Sb, idx, cap, want_count)


def rnnls_sketch_multi(ctx, A, lda, B, ldb, n_raw, d, nrhs, r, seed, instance, SA, ldsa, SB, ldsb, idx) -> None:
    check(lib().rnnls_sketch_multi(ctypes.c_void_p(ctx), ctypes.c_void_p(A), lda, ctypes.c_void_p(B), ldb, n_raw, d,
                                   nrhs, r, seed, instance, ctypes.c_void_p(SA), ldsa, ctypes.c_void_p(SB), ldsb,
                                   ctypes.c_void_p(idx)), "rnnls_sketch_multi")


def rnnls_sketch_shard(ctx, A, lda, b, n_raw, row0, rows, d, r, seed, instance, SA, ldsa, Sb, idx) -> None:
    check(lib().rnnls_sketch_shard(ctypes.c_void_p(ctx), ctypes.c_void_p(A), lda, ctypes.c_void_p(b), n_raw, row0,
                                   rows, d, r, seed, instance, ctypes.c_void_p(SA), ldsa, ctypes.c_void_p(Sb),
                                   ctypes.c_void_p(idx)), "rnnls_sketch_shard")


def rnnls_solve(ctx, SA, ldsa, Sb, r, d, x, info) -> None:
    check(lib().rnnls_solve(ctypes.c_void_p(ctx), ctypes.c_void_p(SA), ldsa, ctypes.c_void_p(Sb), r, d,
                            ctypes.c_void_p(x), ctypes.c_void_p(info)), "rnnls_solve")


def rnnls_solve_f64(ctx, SA, ldsa, Sb, r, d, x, info) -> None:
    check(lib().rnnls_solve_f64(ctypes.c_void_p(ctx), ctypes.c_void_p(SA), ldsa, ctypes.c_void_p(Sb), r, d,
                                ctypes.c_void_p(x), ctypes.c_void_p(info)), "rnnls_solve_f64")


def rnnls_sketch_batched(ctx, jobs, flags: int = 0) -> None:
    arr = (rnnls_sketch_job * len(jobs))(*jobs)
    if flags:
        check(lib().rnnls_sketch_batched_ex(ctypes.c_void_p(ctx), arr, len(jobs), flags), "rnnls_sketch_batched_ex")
    else:
        check(lib().rnnls_sketch_batched(ctypes.c_void_p(ctx), arr, len(jobs)), "rnnls_sketch_batched")


def rnnls_gram(ctx, SA, ldsa, Sb, r, d, Q, colabs) -> None:
    check(lib().rnnls_gram(ctypes.c_void_p(ctx), ctypes.c_void_p(SA), ldsa, ctypes.c_void_p(Sb), r, d,
                           ctypes.c_void_p(Q), ctypes.c_void_p(colabs)), "rnnls_gram")


def rnnls_solve_batched_device(ctx, d_probs, count, max_r, max_d, flags: int = 0) -> None:
    check(lib().rnnls_solve_batched_device(ctypes.c_void_p(ctx), ctypes.c_void_p(d_probs), count, max_r, max_d,
                                           flags), "rnnls_solve_batched_device")


def rnnls_set_tuning(ctx, values: dict) -> None:
    unknown = set(values) - set(TUNING_KNOBS)
    if unknown:
        raise ValueError(f"unknown tuning knobs: {sorted(unknown)}")
    t = rnnls_tuning(**{k: int(v) for k, v in values.items()})
    check(lib().rnnls_set_tuning(ctypes.c_void_p(ctx), ctypes.byref(t)), "rnnls_set_tuning")


def rnnls_get_tuning(ctx) -> dict:
    t = rnnls_tuning()
    check(lib().rnnls_get_tuning(ctypes.c_void_p(ctx), ctypes.byref(t)), "rnnls_get_tuning")
    return {k: getattr(t, k) for k in TUNING_KNOBS}


def rnnls_sketch_csc(ctx, colptr, rowidx, val, b, n_raw, d, r, seed, instance, SA, ldsa, Sb, idx) -> None:
    check(lib().rnnls_sketch_csc(ctypes.c_void_p(ctx), ctypes.c_void_p(colptr), ctypes.c_void_p(rowidx),
                                 ctypes.c_void_p(val), ctypes.c_void_p(b), n_raw, d, r, seed, instance,
                                 ctypes.c_void_p(SA), ldsa, ctypes.c_void_p(Sb), ctypes.c_void_p(idx)),
          "rnnls_sketch_csc")


def rnnls_solve_pg(ctx, SA, ldsa, Sb, r, d, x, info, tol, max_iter) -> None:
    check(lib().rnnls_solve_pg(ctypes.c_void_p(ctx), ctypes.c_void_p(SA), ldsa, ctypes.c_void_p(Sb), r, d,
                               ctypes.c_void_p(x), ctypes.c_void_p(info), tol, max_iter), "rnnls_solve_pg")


def rnnls_solve_multi(ctx, SA, ldsa, SB, ldsb, r, d, nrhs, X, ldx, infos) -> None:
    check(lib().rnnls_solve_multi(ctypes.c_void_p(ctx), ctypes.c_void_p(SA), ldsa, ctypes.c_void_p(SB), ldsb, r, d,
                                  nrhs, ctypes.c_void_p(X), ldx, ctypes.c_void_p(infos)), "rnnls_solve_multi")


def rnnls_solve_batched(ctx, problems, flags: int = 0) -> None:
    arr = (rnnls_problem * len(problems))(*problems)
    check(lib().rnnls_solve_batched(ctypes.c_void_p(ctx), arr, len(problems), flags), "rnnls_solve_batched")


def rnnls_solve_boosted(ctx, A, lda, b, n_raw, d, r, seed, instance0, k, x, resid, best, info) -> None:
    check(lib().rnnls_solve_boosted(ctypes.c_void_p(ctx), ctypes.c_void_p(A), lda, ctypes.c_void_p(b), n_raw, d, r,
                                    seed, instance0, k, ctypes.c_void_p(x), ctypes.c_void_p(resid),
                                    ctypes.c_void_p(best), ctypes.c_void_p(info)), "rnnls_solve_boosted")


def rnnls_residual(ctx, A, lda, b, n, d, x, out) -> None:
    check(lib().rnnls_residual(ctypes.c_void_p(ctx), ctypes.c_void_p(A), lda, ctypes.c_void_p(b), n, d,
                               ctypes.c_void_p(x), ctypes.c_void_p(out)), "rnnls_residual")


def rnnls_profile_begin(ctx, max_launches: int = 4096) -> None:
    check(lib().rnnls_profile_begin(ctypes.c_void_p(ctx), max_launches), "rnnls_profile_begin")


def rnnls_profile_end(ctx) -> dict:
    """{kernel name: (launches, total_ms)} of the launches since rnnls_profile_begin."""
    out = (rnnls_kernel_time * 32)()
    n = ctypes.c_int(0)
    check(lib().rnnls_profile_end(ctypes.c_void_p(ctx), out, 32, ctypes.byref(n)), "rnnls_profile_end")
    return {out[i].name.decode(): (int(out[i].launches), float(out[i].total_ms)) for i in range(n.value)}


def rnnls_strerror(status: int) -> str:
    return lib().rnnls_strerror(status).decode()
