"""GB300-native RandomizedNNLS (Boutsidis & Drineas): the subsampled randomized
Hadamard sketch of a tall [A | b] and the Lawson-Hanson solve on the sketch,
behind the C ABI of include/rnnls.h.

:class:`Context` marshals torch tensors (device memory and streams only) into
the C calls; the same-name raw wrappers live in :mod:`._binding`.
Matrices are column-major: an (n, d) tensor with ``stride(0) == 1``
(e.g. ``torch.empty(d, n, device="cuda").t()``).
"""
from __future__ import annotations

import ctypes
import math

from . import _binding as B
from ._binding import (RNNLS_PREC_BF16X2, RNNLS_PREC_FP32, RNNLS_SAMPLE_BERNOULLI, RNNLS_SAMPLE_IID,  # noqa: F401
                       RNNLSError, rnnls_info,  # noqa: F401
                       rnnls_problem)

INFO_BYTES = ctypes.sizeof(rnnls_info)


def bernoulli_capacity(r: int, n: int) -> int:
    """Row capacity that a Bernoulli-mode sketch output needs (6 sigma above r)."""
    if r >= n:
        return n
    return int(r + math.ceil(6.0 * math.sqrt(r)) + 16)


def padded_n(n_raw: int) -> int:
    n = 1
    while n < n_raw:
        n <<= 1
    return n


def _torch():
    import torch

    return torch


def colmajor(t):
    """Column-major copy (or view) of a 2-D tensor."""
    if t.dim() != 2:
        raise ValueError("expected a matrix")
    if t.stride(0) == 1 and t.stride(1) >= max(t.shape[0], 1):
        return t
    return t.t().contiguous().t()


def _ld(t) -> int:
    return max(int(t.stride(1)), int(t.shape[0]), 1)


def info_dict(raw) -> dict:
    """Decode an rnnls_info held in a uint8 tensor (host or device)."""
    b = bytes(raw.cpu().numpy().tobytes())
    inf = rnnls_info.from_buffer_copy(b[:INFO_BYTES])
    return {k: getattr(inf, k) for k, _ in rnnls_info._fields_}


class Context:
    """One library context bound to a CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None):
        torch = _torch()
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.handle = B.rnnls_create(device, self.stream.cuda_stream)

    def close(self) -> None:
        if getattr(self, "handle", None):
            B.rnnls_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream) -> None:
        self.stream = stream
        B.rnnls_set_stream(self.handle, stream.cuda_stream)

    def set_sketch_sms(self, sms: int) -> None:
        """Cap the SMs the large-n sketch occupies (0: all), leaving the rest to other streams."""
        B.rnnls_set_sketch_sms(self.handle, sms)

    def set_plan_event(self, event) -> None:
        """Record `event` (a torch.cuda.Event, or None) after each sketch's plan launch."""
        B.rnnls_set_plan_event(self.handle, 0 if event is None else event.cuda_event)

    # -- sketch -------------------------------------------------------------------------
    def sketch(self, A, b, r: int, seed: int, instance: int = 0, mode: int = RNNLS_SAMPLE_IID, SA=None, Sb=None,
               idx=None, cap: int | None = None, want_count: bool = True, prec: int = RNNLS_PREC_FP32):
        """SA, Sb, idx and the row count of Alg. 1's sketch (FP32 or FP64 by A's dtype; FP32 data may use
        prec=RNNLS_PREC_BF16X2, the split-precision tensor-core pass)."""
        torch = _torch()
        A = colmajor(A)
        n_raw, d = A.shape
        n = padded_n(n_raw)
        if cap is None:
            cap = r if mode == RNNLS_SAMPLE_IID else bernoulli_capacity(r, n)
        dt = A.dtype
        if SA is None:
            SA = torch.empty((d, cap), dtype=dt, device=A.device).t()
        if Sb is None:
            Sb = torch.empty(cap, dtype=dt, device=A.device)
        if idx is None:
            idx = torch.empty(cap, dtype=torch.int32, device=A.device)
        fn = B.rnnls_sketch if dt == torch.float32 else B.rnnls_sketch_f64
        if dt not in (torch.float32, torch.float64) or b.dtype != dt or SA.dtype != dt or Sb.dtype != dt:
            raise TypeError("A, b, SA, Sb must share dtype float32 or float64")
        if not b.is_contiguous() or not Sb.is_contiguous() or not idx.is_contiguous():
            raise ValueError("b, Sb and idx must be contiguous")
        rows = fn(self.handle, A.data_ptr(), _ld(A), b.data_ptr(), n_raw, d, r, seed, instance, mode | prec,
                  SA.data_ptr(), _ld(SA), Sb.data_ptr(), idx.data_ptr(), cap, want_count)
        return SA, Sb, idx, rows

    def sketch_multi(self, A, Bm, r: int, seed: int, instance: int = 0, SA=None, SB=None, idx=None):
        """SA, SB, idx: one sketch of [A | Bm] for the nrhs columns of Bm (FP32)."""
        torch = _torch()
        A, Bm = colmajor(A), colmajor(Bm)
        n_raw, d = A.shape
        if Bm.shape[0] != n_raw or A.dtype != torch.float32 or Bm.dtype != torch.float32:
            raise ValueError("A and B must be FP32 with the same number of rows")
        nrhs = Bm.shape[1]
        if SA is None:
            SA = torch.empty((d, r), dtype=A.dtype, device=A.device).t()
        if SB is None:
            SB = torch.empty((nrhs, r), dtype=A.dtype, device=A.device).t()
        if idx is None:
            idx = torch.empty(r, dtype=torch.int32, device=A.device)
        B.rnnls_sketch_multi(self.handle, A.data_ptr(), _ld(A), Bm.data_ptr(), _ld(Bm), n_raw, d, nrhs, r, seed,
                              instance, SA.data_ptr(), _ld(SA), SB.data_ptr(), _ld(SB), idx.data_ptr())
        return SA, SB, idx

    def sketch_batched(self, items, prec: int = RNNLS_PREC_FP32):
        """Sketch many FP32 instances together; items: (A, b, r, seed, instance, SA, Sb, idx), outputs preallocated."""
        jobs = []
        for A, b, r, seed, instance, SA, Sb, idx in items:
            A = colmajor(A)
            jobs.append(B.rnnls_sketch_job(A.data_ptr(), _ld(A), b.data_ptr(), A.shape[0], A.shape[1], r, seed, instance,
                                           SA.data_ptr(), _ld(SA), Sb.data_ptr(), idx.data_ptr()))
        B.rnnls_sketch_batched(self.handle, jobs, prec)

    def sketch_shard(self, A_rows, b_rows, n_raw: int, row0: int, r: int, seed: int, instance: int = 0, SA=None,
                     Sb=None, idx=None):
        """This row block's additive part of the full sketch (FP32, iid); A_rows holds rows row0.. only."""
        torch = _torch()
        A_rows = colmajor(A_rows)
        rows, d = A_rows.shape
        if SA is None:
            SA = torch.empty((d, r), dtype=A_rows.dtype, device=A_rows.device).t()
        if Sb is None:
            Sb = torch.empty(r, dtype=A_rows.dtype, device=A_rows.device)
        if idx is None:
            idx = torch.empty(r, dtype=torch.int32, device=A_rows.device)
        B.rnnls_sketch_shard(self.handle, A_rows.data_ptr(), _ld(A_rows), b_rows.data_ptr(), n_raw, row0, rows, d, r,
                              seed, instance, SA.data_ptr(), _ld(SA), Sb.data_ptr(), idx.data_ptr())
        return SA, Sb, idx

    # -- solve ----------------------------------------------------------------------------
    def solve_multi(self, SA, SB, r: int | None = None, X=None, infos=None):
        """X (d x nrhs FP64) and raw infos (nrhs x INFO_BYTES) for targets sharing the sketch SA."""
        torch = _torch()
        SA, SB = colmajor(SA), colmajor(SB)
        r = SA.shape[0] if r is None else r
        d, nrhs = SA.shape[1], SB.shape[1]
        if X is None:
            X = torch.empty((nrhs, d), dtype=torch.float64, device=SA.device).t()
        if infos is None:
            infos = torch.zeros((nrhs, INFO_BYTES), dtype=torch.uint8, device=SA.device)
        B.rnnls_solve_multi(self.handle, SA.data_ptr(), _ld(SA), SB.data_ptr(), _ld(SB), r, d, nrhs, X.data_ptr(),
                            _ld(X), infos.data_ptr())
        return X, infos

    def solve(self, SA, Sb, r: int | None = None, x=None, info=None):
        """x = argmin_{x>=0} ||SA x - Sb||^2 (Lawson-Hanson); returns (x, info bytes)."""
        torch = _torch()
        SA = colmajor(SA)
        rr = SA.shape[0] if r is None else r
        d = SA.shape[1]
        if x is None:
            x = torch.empty(d, dtype=torch.float64, device=SA.device)
        if info is None:
            info = torch.zeros(INFO_BYTES, dtype=torch.uint8, device=SA.device)
        fn = B.rnnls_solve if SA.dtype == torch.float32 else B.rnnls_solve_f64
        fn(self.handle, SA.data_ptr(), _ld(SA), Sb.data_ptr(), rr, d, x.data_ptr(), info.data_ptr())
        return x, info

    def get_tuning(self) -> dict:
        """The context's launch-shape choices (rnnls_tuning; 0 = built-in default)."""
        return B.rnnls_get_tuning(self.handle)

    def set_tuning(self, values: dict) -> None:
        """Replace the context's launch-shape choices (missing knobs: default)."""
        B.rnnls_set_tuning(self.handle, values)

    def sketch_csc(self, colptr, rowidx, val, b, n_raw: int, d: int, r: int, seed: int, instance: int = 0,
                   SA=None, Sb=None, idx=None):
        """Sketch of a sparse A in compressed columns (device int64 colptr, int32 rowidx,
        float32 val) with a dense b; returns (SA, Sb, idx)."""
        torch = _torch()
        dev = b.device
        if SA is None:
            SA = torch.empty((d, r), dtype=torch.float32, device=dev).t()
        if Sb is None:
            Sb = torch.empty(r, dtype=torch.float32, device=dev)
        if idx is None:
            idx = torch.empty(r, dtype=torch.int32, device=dev)
        B.rnnls_sketch_csc(self.handle, colptr.data_ptr(), rowidx.data_ptr() if rowidx.numel() else 0,
                           val.data_ptr() if val.numel() else 0, b.data_ptr(), n_raw, d, r, seed, instance,
                           SA.data_ptr(), _ld(SA), Sb.data_ptr(), idx.data_ptr())
        return SA, Sb, idx

    def solve_pg(self, SA, Sb, r: int | None = None, x=None, info=None, tol: float = 1e-12, max_iter: int = 50000):
        """x ~ argmin_{x>=0} ||SA x - Sb||^2 by accelerated projected gradient on the
        quadratic-programming form (d up to 8192); returns (x, info bytes)."""
        torch = _torch()
        SA = colmajor(SA)
        rr = SA.shape[0] if r is None else r
        d = SA.shape[1]
        if x is None:
            x = torch.empty(d, dtype=torch.float64, device=SA.device)
        if info is None:
            info = torch.zeros(INFO_BYTES, dtype=torch.uint8, device=SA.device)
        B.rnnls_solve_pg(self.handle, SA.data_ptr(), _ld(SA), Sb.data_ptr(), rr, d, x.data_ptr(), info.data_ptr(),
                         tol, max_iter)
        return x, info

    def gram(self, SA, Sb, r: int | None = None, Q=None, colabs=None):
        """Sketch moments Q = [SA | Sb]'[SA | Sb] ((d+1) x (d+1), FP64) and the
        column 1-norms of SA; returns (Q, colabs), device tensors."""
        torch = _torch()
        SA = colmajor(SA)
        rr = SA.shape[0] if r is None else r
        d = SA.shape[1]
        if Q is None:
            Q = torch.empty((d + 1, d + 1), dtype=torch.float64, device=SA.device)
        if colabs is None:
            colabs = torch.empty(d, dtype=torch.float64, device=SA.device)
        B.rnnls_gram(self.handle, SA.data_ptr(), _ld(SA), Sb.data_ptr(), rr, d, Q.data_ptr(), colabs.data_ptr())
        return Q, colabs

    def solve_batched(self, problems):
        """problems: list of (SA, Sb, x, info) tensors; FP32 sketches."""
        descs = []
        for SA, Sb, x, info in problems:
            SA = colmajor(SA)
            descs.append(rnnls_problem(SA.data_ptr(), _ld(SA), Sb.data_ptr(), SA.shape[0], SA.shape[1], x.data_ptr(),
                                       info.data_ptr() if info is not None else None))
        B.rnnls_solve_batched(self.handle, descs, 0)

    def solve_boosted(self, A, b, r: int, k: int, seed: int, instance0: int = 0, x=None, resid=None, best=None,
                      info=None):
        """k runs of Alg. 1 (instances instance0 .. instance0 + k - 1), the one with the smallest
        ||A x_j - b||^2 kept; returns (x, resid (k), best (1, int32), info bytes), all on the device."""
        torch = _torch()
        A = colmajor(A)
        n, d = A.shape
        dev = A.device
        if x is None:
            x = torch.empty(d, dtype=torch.float64, device=dev)
        if resid is None:
            resid = torch.empty(k, dtype=torch.float64, device=dev)
        if best is None:
            best = torch.empty(1, dtype=torch.int32, device=dev)
        if info is None:
            info = torch.zeros(INFO_BYTES, dtype=torch.uint8, device=dev)
        B.rnnls_solve_boosted(self.handle, A.data_ptr(), _ld(A), b.data_ptr(), n, d, r, seed, instance0, k,
                              x.data_ptr(), resid.data_ptr(), best.data_ptr(), info.data_ptr())
        return x, resid, best, info

    def residual(self, A, b, x, out=None):
        """||A x - b||^2 on the full data (FP64 accumulation), a 1-element device tensor."""
        torch = _torch()
        A = colmajor(A)
        if out is None:
            out = torch.empty(1, dtype=torch.float64, device=A.device)
        B.rnnls_residual(self.handle, A.data_ptr(), _ld(A), b.data_ptr(), A.shape[0], A.shape[1], x.data_ptr(),
                         out.data_ptr())
        return out

    def randomized_nnls(self, A, b, r: int, seed: int, instance: int = 0, mode: int = RNNLS_SAMPLE_IID):
        """Alg. 1 end to end on device tensors: sketch, then Lawson-Hanson."""
        SA, Sb, idx, rows = self.sketch(A, b, r, seed, instance, mode)
        x, info = self.solve(SA[:rows], Sb[:rows], r=rows)
        return x, info, (SA, Sb, idx, rows)


def lib_path() -> str:
    return B.lib_path()
