"""Shared helpers of the GPU tests: column-major tensors between numpy and torch, error norms."""
import numpy as np


def to_dev(a: np.ndarray, dtype=None):
    """numpy column-major (Fortran) array -> contiguous CUDA tensor with the same memory."""
    import torch
    a = np.asfortranarray(a if dtype is None else a.astype(dtype))
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda()


def from_dev(t) -> np.ndarray:
    """CUDA tensor holding a column-major tensor -> numpy Fortran array with the label shape."""
    return np.asfortranarray(t.cpu().numpy().T)


def normwise(x, ref):
    ref = np.asarray(ref, dtype=np.float64)
    d = np.abs(np.asarray(x, dtype=np.float64) - ref)
    return float(d.max() / max(np.abs(ref).max(), 1e-300))


def maxabs(x, ref):
    return float(np.abs(np.asarray(x, dtype=np.float64) - np.asarray(ref, dtype=np.float64)).max())


def empty_like_labels(extents, dtype):
    import torch
    return torch.zeros(tuple(reversed([int(e) for e in extents])), dtype=dtype, device="cuda")
