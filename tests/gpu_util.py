"""Helpers shared by the GPU parity tests (test infrastructure)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1406_5369_gb300 import build as b
    b.build()
    return torch


def rel_err(a, b):
    """max |a - b| / max |b| (max |b| floored at tiny)."""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def interior(a):
    return a[(slice(1, -1),) * a.ndim]


def zero_boundary(a):
    out = np.zeros_like(a)
    out[(slice(1, -1),) * a.ndim] = interior(a)
    return out


# Storage-precision tolerances for operator parity (max-abs error over max-abs
# value). FP64: a few ulps of rounding-order difference (FMA contraction and
# summation order) over the handful of operations per node. FP32: ~2^-24 per
# operation over up to 2 sweeps. BF16: one rounding to 8 significant bits.
OP_TOL = {"fp64": 1e-13, "fp32_dc": 2e-5, "bf16_dc": 2e-2}
