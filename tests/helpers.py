"""Shared helpers of the GPU parity tests."""
import numpy as np
import pytest


def normwise_rel(a, ref) -> float:
    """max |a - ref| / max |ref| (the normwise infinity relative error)."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.abs(ref).max()
    if den == 0:
        return float(np.abs(a).max())
    return float(np.abs(a - ref).max() / den)


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch


def dev(t, torch):
    return torch.from_numpy(np.ascontiguousarray(t, dtype=np.float32)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)
