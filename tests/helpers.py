"""Shared helpers of the GPU tests: column-major tensors between numpy and torch, error norms."""
import numpy as np


def to_dev(a: np.ndarray, dtype=None, device="cuda"):
    """numpy column-major (Fortran) array -> contiguous torch tensor with the same memory."""
    import torch
    a = np.asarray(a if dtype is None else np.asarray(a).astype(dtype))
    if a.ndim == 0:
        return torch.from_numpy(a.reshape(())).to(device)
    a = np.asfortranarray(a)
    return torch.from_numpy(np.ascontiguousarray(a.T)).to(device)


def from_dev(t) -> np.ndarray:
    """torch tensor holding a column-major tensor -> numpy Fortran array with the label shape."""
    a = t.cpu().numpy()
    if a.ndim == 0:
        return a.copy()
    return np.asfortranarray(a.T)


def same_bits(x: np.ndarray, y: np.ndarray) -> bool:
    return x.shape == y.shape and x.dtype == y.dtype and x.tobytes(order="F") == y.tobytes(order="F")


def normwise(x, ref):
    ref = np.asarray(ref, dtype=np.float64)
    d = np.abs(np.asarray(x, dtype=np.float64) - ref)
    return float(d.max() / max(np.abs(ref).max(), 1e-300))


def maxabs(x, ref):
    return float(np.abs(np.asarray(x, dtype=np.float64) - np.asarray(ref, dtype=np.float64)).max())


def empty_like_labels(extents, dtype, device="cuda"):
    import torch
    return torch.zeros(tuple(reversed([int(e) for e in extents])), dtype=dtype, device=device)
