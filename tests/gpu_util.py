"""Helpers shared by the GPU tests: device buffers from torch, the current
stream, and the library handle."""
import numpy as np


def torch_mod():
    import torch
    return torch


def stream():
    torch = torch_mod()
    return torch.cuda.current_stream().cuda_stream


def to_dev(a, dtype=None):
    """Column-major host block -> CUDA tensor holding the same column-major
    memory (returned as the transposed view of an (m, N) row-major tensor)."""
    torch = torch_mod()
    a = np.asarray(a)
    if dtype is not None:
        a = a.astype(dtype)
    if a.ndim == 1:
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    t = torch.from_numpy(np.ascontiguousarray(a.T)).cuda()  # (m, N) row-major
    return t


def from_dev(t, shape=None):
    """Inverse of to_dev for blocks: (m, N) row-major tensor -> (N, m) numpy."""
    torch = torch_mod()
    torch.cuda.synchronize()
    x = t.detach().cpu().numpy()
    if x.ndim == 2:
        return np.asfortranarray(x.T)
    return x


def empty(N, m, dtype):
    torch = torch_mod()
    td = {np.float64: torch.float64, np.float32: torch.float32}[dtype]
    return torch.zeros((m, N), dtype=td, device="cuda")
