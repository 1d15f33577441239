"""Helpers of the GPU tests: device availability and relative errors."""
import numpy as np
import pytest


def cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def need_gpu():
    if not cuda_ok():
        pytest.skip("no CUDA device")
