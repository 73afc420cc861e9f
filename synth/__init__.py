"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module holds no multigrid arithmetic: it only draws numbers and lays
them out on node-based grids, so that the oracle (``oracle/``) and the GPU
library see bit-identical right-hand sides, coefficients and initial guesses.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: draw ``i`` of stream ``seed`` is ``mix(seed + (i + 1) * GAMMA)``.
Uniforms take the top 53 bits; normals use the Box-Muller transform on
consecutive pairs of uniforms.

Grid convention (node-based, as in the paper's Layer 2 ``field@nodes``): a
level with ``n = 2**m + 1`` nodes per dimension spans [0, 1]^dim with
spacing ``h = 1/(n-1)``; arrays have shape ``(n,)*dim`` in C order with x
fastest (``u[j, i]`` in 2D, ``u[k, j, i]`` in 3D); boundary nodes are the
first and last index along every axis.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22

# Seeds for the named workloads: workload i uses WORKLOAD_SEED_BASE + i and,
# inside a batch, problem p uses (seed ^ p).
WORKLOAD_SEED_BASE = 0x5EED0000


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Draws ``start .. start+count-1`` of the SplitMix64 stream ``seed`` (uint64)."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GAMMA
    return _mix(z)


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """U[0, 1) doubles from the top 53 bits of each draw."""
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _fill(out_flat: np.ndarray, fn) -> None:
    total = out_flat.size
    for s in range(0, total, _CHUNK):
        e = min(total, s + _CHUNK)
        out_flat[s:e] = fn(s, e - s)


def uniform(seed: int, shape, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    out = np.empty(shape, dtype=np.float64)
    _fill(out.reshape(-1), lambda s, c: lo + (hi - lo) * uniform01(seed, c, s))
    return out


def normal(seed: int, shape) -> np.ndarray:
    """Standard normals: Box-Muller on the uniform pair (2i, 2i+1)."""
    out = np.empty(shape, dtype=np.float64)

    def block(s, c):
        u = uniform01(seed, 2 * c, 2 * s)
        u1, u2 = u[0::2], u[1::2]
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)

    _fill(out.reshape(-1), block)
    return out


def _zero_boundary(a: np.ndarray) -> np.ndarray:
    for ax in range(a.ndim):
        idx = [slice(None)] * a.ndim
        idx[ax] = 0
        a[tuple(idx)] = 0.0
        idx[ax] = -1
        a[tuple(idx)] = 0.0
    return a


def check_size(dim: int, n: int) -> int:
    """Returns m for n = 2**m + 1 (m >= 1), else raises ValueError."""
    if dim not in (2, 3):
        raise ValueError(f"dim must be 2 or 3, got {dim}")
    m = (n - 1).bit_length() - 1
    if n < 3 or (1 << m) + 1 != n:
        raise ValueError(f"n must be 2**m + 1 with m >= 1, got {n}")
    return m


def coords(n: int) -> np.ndarray:
    return np.arange(n, dtype=np.float64) / (n - 1)


def sine_rhs(dim: int, n: int) -> np.ndarray:
    """f = dim * pi^2 * prod_d sin(pi x_d): the right-hand side whose continuous
    solution of -Laplace(u) = f with u = 0 on the boundary is prod_d sin(pi x_d)."""
    check_size(dim, n)
    s = np.sin(math.pi * coords(n))
    s[0] = s[-1] = 0.0
    if dim == 2:
        f = np.multiply.outer(s, s)
    else:
        f = np.multiply.outer(np.multiply.outer(s, s), s)
    return np.ascontiguousarray(dim * math.pi ** 2 * f)


def sine_solution(dim: int, n: int) -> np.ndarray:
    """prod_d sin(pi x_d) at the nodes (the continuous solution for sine_rhs)."""
    return sine_rhs(dim, n) / (dim * math.pi ** 2)


def uniform_rhs(dim: int, n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """i.i.d. U[lo, hi] at interior nodes, 0 on the boundary."""
    check_size(dim, n)
    return _zero_boundary(uniform(seed, (n,) * dim, lo, hi))


def normal_rhs(dim: int, n: int, seed: int) -> np.ndarray:
    """i.i.d. N(0, 1) at interior nodes, 0 on the boundary."""
    check_size(dim, n)
    return _zero_boundary(normal(seed, (n,) * dim))


def lognormal_k(dim: int, n: int, seed: int, mu: float = 0.0, sigma: float = 1.0) -> np.ndarray:
    """Node (dual-cell) diffusivities k = exp(mu + sigma * z), z ~ N(0, 1), at every node."""
    check_size(dim, n)
    return np.exp(mu + sigma * normal(seed, (n,) * dim))


def random_u0(dim: int, n: int, seed: int) -> np.ndarray:
    """Initial guess U[0, 1) at interior nodes, 0 on the boundary."""
    check_size(dim, n)
    return _zero_boundary(uniform(seed, (n,) * dim, 0.0, 1.0))


def batch_levels(count: int, seed: int, m_lo: int = 5, m_hi: int = 10) -> np.ndarray:
    """m ~ U{m_lo..m_hi} for each of ``count`` problems (grid n = 2**m + 1)."""
    u = uniform01(seed, count)
    return (m_lo + np.floor(u * (m_hi - m_lo + 1))).astype(np.int64)


def serving_requests(count: int, seed: int, rate_per_s: float = 2000.0,
                     frac_2d: float = 0.7, m2d=(6, 12), m3d=(5, 8),
                     tols=(1e-6, 1e-10)):
    """A Poisson arrival stream of solve requests.

    Returns a list of dicts with arrival time (s), dim, n, tol and a per-request
    seed. Each request consumes five uniforms: inter-arrival time (exponential
    with the given rate), dimension, level exponent (uniform over the integer
    range, i.e. log-uniform over grid sizes 2**m + 1), tolerance and a seed.
    """
    u = uniform01(seed, 5 * count).reshape(count, 5)
    t = 0.0
    out = []
    for r in range(count):
        t += -math.log1p(-u[r, 0]) / rate_per_s
        dim = 2 if u[r, 1] < frac_2d else 3
        lo, hi = m2d if dim == 2 else m3d
        m = lo + int(u[r, 2] * (hi - lo + 1))
        tol = tols[0] if u[r, 3] < 0.5 else tols[1]
        out.append({"id": r, "t": t, "dim": dim, "n": (1 << m) + 1, "tol": tol,
                    "seed": (seed ^ (r + 1)) & 0xFFFFFFFF})
    return out


# ---------------------------------------------------------------- torch (device) generation
# The same counter-based SplitMix64 in torch int64 arithmetic, so that large
# inputs can be drawn where they are used (e.g. on the GPU) with bit-identical
# values to the numpy functions above. int64 products wrap modulo 2^64; right
# shifts are made logical by masking off the copied sign bits.

def _t_const(x):
    return x - (1 << 64) if x >= (1 << 63) else x


_T_GAMMA = _t_const(0x9E3779B97F4A7C15)
_T_M1 = _t_const(0xBF58476D1CE4E5B9)
_T_M2 = _t_const(0x94D049BB133111EB)


def _t_shr(z, k):
    return (z >> k) & ((1 << (64 - k)) - 1)


def torch_seed(seed: int) -> int:
    """A seed as the signed 64-bit integer the torch generators add: the value
    to store in a 0-dim int64 tensor passed as `seed` (e.g. one a CUDA graph
    of a generator reads)."""
    return _t_const(seed & 0xFFFFFFFFFFFFFFFF)


def torch_splitmix64(seed, count: int, start: int = 0, device="cpu"):
    """seed: an int, or a 0-dim int64 tensor holding torch_seed(seed)."""
    import torch
    idx = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    z = idx * _T_GAMMA + (seed if isinstance(seed, torch.Tensor) else torch_seed(seed))
    z = (z ^ _t_shr(z, 30)) * _T_M1
    z = (z ^ _t_shr(z, 27)) * _T_M2
    return z ^ _t_shr(z, 31)


def torch_uniform01(seed: int, count: int, start: int = 0, device="cpu"):
    import torch
    z = torch_splitmix64(seed, count, start, device)
    return _t_shr(z, 11).to(torch.float64) * (2.0 ** -53)


def torch_uniform(seed: int, shape, lo: float = -1.0, hi: float = 1.0, device="cpu"):
    count = 1
    for s in shape:
        count *= s
    out = lo + (hi - lo) * torch_uniform01(seed, count, 0, device)
    return out.reshape(tuple(shape))


def _t_zero_boundary(a):
    for ax in range(a.dim()):
        a.select(ax, 0).zero_()
        a.select(ax, a.shape[ax] - 1).zero_()
    return a


def torch_uniform_rhs(dim: int, n: int, seed: int, lo: float = -1.0, hi: float = 1.0, device="cpu"):
    """Same values as uniform_rhs, drawn with torch on `device`."""
    check_size(dim, n)
    return _t_zero_boundary(torch_uniform(seed, (n,) * dim, lo, hi, device)).contiguous()


def torch_lognormal_k(dim: int, n: int, seed: int, mu: float = 0.0, sigma: float = 1.0, device="cpu"):
    """k = exp(mu + sigma z), z by Box-Muller on the uniform pair (2i, 2i+1), as
    lognormal_k; the uniforms are bit-identical, the transcendental functions
    are the device's (equal to numpy's to a few ulps)."""
    import torch
    check_size(dim, n)
    count = n ** dim
    u = torch_uniform01(seed, 2 * count, 0, device)
    z = torch.sqrt(-2.0 * torch.log1p(-u[0::2])) * torch.cos(2.0 * math.pi * u[1::2])
    return torch.exp(mu + sigma * z).reshape((n,) * dim).contiguous()
