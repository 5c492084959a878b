"""Shared set-up of the GPU tests: build once, load the binding, torch device buffers."""
import numpy as np
import pytest


def gpu_modules():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_11801_gb300 import build as B
    B.build()
    from paper_2312_11801_gb300 import usbs as U
    U.load()
    return torch, U


def bulk_dtype(torch, precision):
    return torch.float64 if precision == 0 else torch.float32


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
