"""Helpers for the GPU parity tests (host <-> device marshalling only)."""
import numpy as np


def dev_colmajor(a: np.ndarray, dtype=None):
    """Column-major CUDA tensor holding the bytes of `a` (converted to dtype)."""
    import torch

    a = np.asarray(a)
    if dtype is not None:
        a = a.astype(dtype)
    src = torch.from_numpy(np.ascontiguousarray(a.T))
    # (d, n) row-major == (n, d) column-major; torch.empty fixes the leading
    # dimension at n even when d == 1
    t = torch.empty(src.shape, dtype=src.dtype, device="cuda")
    t.copy_(src)
    return t.t()


def dev_vec(v: np.ndarray, dtype=None):
    import torch

    v = np.asarray(v)
    if dtype is not None:
        v = v.astype(dtype)
    return torch.from_numpy(np.ascontiguousarray(v)).cuda()


def host(t) -> np.ndarray:
    return t.detach().cpu().numpy()


def rel_fro(got: np.ndarray, want: np.ndarray) -> float:
    den = np.linalg.norm(want)
    return float(np.linalg.norm(np.asarray(got, dtype=np.float64) - want) / (den if den > 0 else 1.0))
