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


def error_vs_converged_oracle(u, f, maxit=40, tol=1e-13, **hier_kw):
    """Relative l2 error of a solution u against the oracle's FP64 solution of
    the same problem (Dirichlet 0, constant stencil), converged from zero on
    every host core (the oracle's OpenMP build, bitwise its serial result) to
    `tol` or `maxit` cycles; plus the guaranteed bound
    ||u - u*|| <= (||f - A u|| + ||f - A u*||) / lambda_min(A),
    lambda_min = d (4/h^2) sin^2(pi h/2). Returns (rel_l2, bound_rel_l2, oracle_relres)."""
    import math
    import oracle
    oracle.set_threads(oracle.host_cores())
    dim, n = u.ndim, u.shape[0]
    H = oracle.Hierarchy(dim, n, mt=True, **hier_kw)
    H.set_rhs(f)
    rho = H.solve(tol, maxit)
    us = H.get_u()
    del H
    h = 1.0 / (n - 1)
    lam = dim * 4.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2
    r_u = oracle.norm(oracle.residual(u, f, mt=True), mt=True)
    r_s = oracle.norm(oracle.residual(us, f, mt=True), mt=True)
    d = u - us
    nu = float(np.sqrt(np.sum(us * us)))
    return float(np.sqrt(np.sum(d * d))) / nu, (r_u + r_s) / lam / nu, float(rho[-1])
