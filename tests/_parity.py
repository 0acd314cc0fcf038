"""Shared helpers of the parity tests: the error metric and tensor moves."""
import numpy as np


def rel_err(a, b):
    """max_i |a_i - b_i| / max(|b_i|, 1e-3 max_j |b_j|)."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    assert a.shape == b.shape
    if b.size == 0:
        return 0.0
    floor = 1e-3 * np.max(np.abs(b))
    den = np.maximum(np.abs(b), floor if floor > 0 else 1e-300)
    return float(np.max(np.abs(a - b) / den))


def dev(a, dtype=None):
    import torch
    a = np.asarray(a)
    if dtype is None:
        dtype = {np.dtype(np.float64): torch.float64, np.dtype(np.int32): torch.int32,
                 np.dtype(np.int64): torch.int64}[a.dtype]
    return torch.as_tensor(a, dtype=dtype, device="cuda:0").contiguous()


def host(t):
    return t.detach().cpu().numpy()
