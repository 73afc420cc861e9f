"""Local Fourier analysis (LFA) of the node-based two-grid cycle, for choosing
the smoother, its relaxation weight and the sweep counts.

Sec. 2.3 names LFA as the tool that rates the Layer-3 component choices of the
feature model, and Sec. 5 sets choosing them automatically as the goal. This
module predicts the two-grid convergence factor of a configuration from
Fourier symbols (host-side numpy; no GPU work) and ``choose`` ranks candidate
configurations by predicted cost to a tolerance. ``autotune.lfa_choice`` is
the autotuner's entry point.

Setting: the operator -sum_d c_d d^2/dx_d^2 on an infinite node-based grid,
coarsening by 2 in every direction, full-weighting restriction, bi-/trilinear
interpolation, the rediscretised coarse operator, and omega-Jacobi or
omega red-black Gauss-Seidel (red = even i+j[+k], first). A low frequency
theta in [-pi/2, pi/2)^d and its 2^d coarsening harmonics theta + pi*alpha,
alpha in {0,1}^d, span an invariant space of the two-grid operator; on it
(with h = 1)
  A_alpha   = sum_d c_d (2 - 2 cos theta_alpha,d)          (fine symbol),
  A_H       = sum_d c_d (2 - 2 cos 2 theta_d) / 4           (coarse symbol),
  r_alpha   = prod_d (1 + cos theta_alpha,d) / 2            (restriction),
  p_alpha   = r_alpha                                       (interpolation),
  K         = I - p A_H^{-1} r^T diag(A)                    (coarse correction),
  Jacobi    S = I + D,  D = diag(-omega A_alpha / diag),  diag = 2 sum_d c_d,
  red-black S = (I + (I - X) D / 2)(I + (I + X) D / 2), X the pairing
              alpha <-> alpha xor (1,...,1) (multiplying by the colour
              pattern (-1)^(i+j+k) shifts every frequency by pi in each
              direction),
and the two-grid factor is the supremum over theta != 0 of the spectral
radius of S^nu2 K S^nu1.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

SMOOTHERS = ("rbgs", "jacobi")


def _thetas(dim, m):
    # a cell-centred sample of [-pi/2, pi/2)^dim: never hits theta = 0
    t = -math.pi / 2 + (np.arange(m) + 0.5) * math.pi / m
    grids = np.meshgrid(*([t] * dim), indexing="ij")
    return np.stack([g.reshape(-1) for g in grids], axis=1)  # (M, dim)


def _smoother(dim, smoother, omega, A, c):
    """Smoothing operator on the harmonic space, (M, H, H)."""
    H = 2 ** dim
    D = -omega * A / (2.0 * np.sum(c))  # (M, H)
    Dm = D[:, None, :] * np.eye(H)[None]  # diag(D) as (M, H, H)
    if smoother == "jacobi":
        return np.eye(H)[None] + Dm
    if smoother == "rbgs":
        X = np.zeros((H, H))
        for a in range(H):
            X[a, H - 1 - a] = 1.0  # index of alpha xor (1,...,1) in the product order
        red = np.eye(H)[None] + 0.5 * (np.eye(H) + X)[None] @ Dm
        black = np.eye(H)[None] + 0.5 * (np.eye(H) - X)[None] @ Dm
        return black @ red
    raise ValueError(f"unknown smoother {smoother!r}")


def _symbols(dim, th, c):
    alphas = np.array(list(itertools.product((0, 1), repeat=dim)), dtype=np.float64)  # (H, dim)
    tha = th[:, None, :] + math.pi * alphas[None, :, :]  # (M, H, dim)
    A = np.sum(c * (2.0 - 2.0 * np.cos(tha)), axis=2)  # (M, H)
    return tha, A


def two_grid_operators(dim, smoother, omega, nu1, nu2, c=(1.0, 1.0, 1.0), m=32, th=None):
    """The (M, 2^dim, 2^dim) two-grid matrices at M = m^dim low frequencies
    (or at the given (M, dim) frequencies th)."""
    c = np.asarray(list(c)[:dim], dtype=np.float64)
    if th is None:
        th = _thetas(dim, m)
    H = 2 ** dim
    tha, A = _symbols(dim, th, c)
    AH = np.sum(c * (2.0 - 2.0 * np.cos(2.0 * th)), axis=1) / 4.0  # (M,)
    r = np.prod((1.0 + np.cos(tha)) / 2.0, axis=2)  # (M, H)
    K = np.eye(H)[None] - (r[:, :, None] * r[:, None, :] * A[:, None, :]) / AH[:, None, None]
    S = _smoother(dim, smoother, omega, A, c)
    return th, np.linalg.matrix_power(S, nu2) @ K @ np.linalg.matrix_power(S, nu1)


def cc_two_grid_operators(dim, smoother, omega, nu1, nu2, c=(1.0, 1.0, 1.0), m=32, th=None):
    """Two-grid matrices for cell-centred grids (the mg_cc.h operator with
    sigma h^2 -> 0): mean-of-children restriction and constant interpolation.
    With the cell centres x_i = i + 1/2 and the coarse centres X = 2I + 1 (in
    fine cells), the restriction maps the harmonic theta + pi*alpha to the
    coarse frequency 2 theta with the factor prod_d cos(theta_d / 2)
    (alpha_d = 0) or sin(theta_d / 2) (alpha_d = 1), and constant
    interpolation has the same components, so p = r as for the node-based
    transfers but one order lower (no square: the node-based factor is
    prod_d cos^2)."""
    c = np.asarray(list(c)[:dim], dtype=np.float64)
    if th is None:
        th = _thetas(dim, m)
    H = 2 ** dim
    _, A = _symbols(dim, th, c)
    AH = np.sum(c * (2.0 - 2.0 * np.cos(2.0 * th)), axis=1) / 4.0
    alphas = np.array(list(itertools.product((0, 1), repeat=dim)), dtype=np.float64)
    half = th / 2.0
    r = np.prod(np.where(alphas[None, :, :] == 0, np.cos(half)[:, None, :], np.sin(half)[:, None, :]), axis=2)
    K = np.eye(H)[None] - (r[:, :, None] * r[:, None, :] * A[:, None, :]) / AH[:, None, None]
    S = _smoother(dim, smoother, omega, A, c)
    return th, np.linalg.matrix_power(S, nu2) @ K @ np.linalg.matrix_power(S, nu1)


def smoothing_operators(dim, smoother, omega, nu, c=(1.0, 1.0, 1.0), m=32, th=None):
    """Ideal coarse-grid correction: Q S^nu, Q the projection onto the high
    harmonics (alpha != 0)."""
    c = np.asarray(list(c)[:dim], dtype=np.float64)
    if th is None:
        th = _thetas(dim, m)
    H = 2 ** dim
    _, A = _symbols(dim, th, c)
    Q = np.eye(H)
    Q[0, 0] = 0.0
    return th, Q[None] @ np.linalg.matrix_power(_smoother(dim, smoother, omega, A, c), nu)


def _sup(ops, dim, m, refine):
    """Largest spectral radius of ops(th) over a sample of m^dim low
    frequencies, then `refine` rounds of local search (a 5^dim stencil of half
    the previous spacing) around the best few frequencies, kept inside
    [-pi/2, pi/2]^dim and away from theta = 0, where the coarse symbol
    vanishes."""
    th = _thetas(dim, m)
    rho = np.max(np.abs(np.linalg.eigvals(ops(th))), axis=1)
    step = math.pi / m
    best = th[np.argsort(rho)[-4:]]
    top = float(np.max(rho))
    offs = np.array(list(itertools.product((-1.0, -0.5, 0.0, 0.5, 1.0), repeat=dim)))
    for _ in range(refine):
        step /= 2.0
        cand = (best[:, None, :] + step * offs[None, :, :]).reshape(-1, dim)
        cand = np.clip(cand, -math.pi / 2, math.pi / 2)
        cand = cand[np.max(np.abs(cand), axis=1) > 1e-6]
        rc = np.max(np.abs(np.linalg.eigvals(ops(cand))), axis=1)
        top = max(top, float(np.max(rc)))
        best = cand[np.argsort(rc)[-4:]]
    return top


def two_grid_factor(dim, smoother, omega, nu1, nu2, c=(1.0, 1.0, 1.0), m=None, refine=4):
    """Predicted asymptotic convergence factor per two-grid cycle."""
    m = m or (32 if dim == 2 else 12)
    return _sup(lambda th: two_grid_operators(dim, smoother, omega, nu1, nu2, c, th=th)[1], dim, m, refine)


def cc_two_grid_factor(dim, smoother, omega, nu1, nu2, c=(1.0, 1.0, 1.0), m=None, refine=4):
    """Predicted two-grid factor on cell-centred grids (cell-centred restriction,
    constant interpolation). V-cycles with these transfers converge more slowly
    than the two-grid cycle and degrade with the number of levels (transfer
    orders 1 + 1 do not exceed the operator's 2); the prediction ranks
    smoothers, it does not bound the V-cycle."""
    m = m or (32 if dim == 2 else 12)
    return _sup(lambda th: cc_two_grid_operators(dim, smoother, omega, nu1, nu2, c, th=th)[1], dim, m, refine)


def smoothing_factor(dim, smoother, omega, nu=1, c=(1.0, 1.0, 1.0), m=None, refine=4):
    """Smoothing factor per sweep (ideal coarse-grid correction)."""
    m = m or (32 if dim == 2 else 12)
    top = _sup(lambda th: smoothing_operators(dim, smoother, omega, nu, c, th=th)[1], dim, m, refine)
    return top ** (1.0 / nu)


def cycle_words(dim, nu1, nu2):
    """Operator-model traffic of one V(nu1, nu2) cycle in words per fine node:
    per level 3 per sweep, 3 for the residual, 1 + 2^-d for the restriction,
    2^-d for the zero start, 2 + 2^-d for interpolation and correction,
    summed over the levels (factor 2^d / (2^d - 1))."""
    q = 2.0 ** -dim
    return (3.0 * (nu1 + nu2) + 3.0 + (1.0 + q) + q + (2.0 + q)) / (1.0 - q)


def choose(dim, c=(1.0, 1.0, 1.0), tol=1e-10, smoothers=SMOOTHERS, omegas=None, nus=None, grid="node"):
    """Ranks configurations by predicted cost to reduce the residual by `tol`:
    cycles = ceil(log tol / log rho_TG) times cycle_words. grid: "node"
    (node-based transfers) or "cell" (cell-centred transfers). Returns the
    ranked list of dicts (smoother, omega, nu1, nu2, rho, cycles, words)."""
    factor = {"node": two_grid_factor, "cell": cc_two_grid_factor}[grid]
    if omegas is None:
        omegas = {"rbgs": [1.0, 1.05, 1.1, 1.15, 1.2, 1.25, 1.3],
                  "jacobi": [0.5, 0.6, 0.7, 0.75, 0.8, 0.85, 0.9, 1.0]}
    if nus is None:
        nus = [(1, 0), (1, 1), (2, 1), (1, 2), (2, 2), (3, 2), (3, 3)]
    out = []
    for sm in smoothers:
        for om in omegas[sm]:
            for nu1, nu2 in nus:
                rho = factor(dim, sm, om, nu1, nu2, c)
                if not rho < 1.0:
                    continue
                cycles = max(1, math.ceil(math.log(tol) / math.log(max(rho, 1e-300))))
                out.append({"smoother": sm, "omega": om, "nu1": nu1, "nu2": nu2, "rho": rho, "cycles": cycles,
                            "words": cycles * cycle_words(dim, nu1, nu2)})
    out.sort(key=lambda d: (d["words"], d["rho"]))
    return out
