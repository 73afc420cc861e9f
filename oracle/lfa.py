"""Local Fourier analysis (LFA) of the two-grid method: TEST INFRASTRUCTURE ONLY.

Sec. 2.3 names LFA (Wienands & Joppich) as the tool that predicts multigrid
convergence factors for the Layer-3 component choices. This module computes
those predictions for the constant-coefficient operator -sum_d c_d d^2/dx_d^2
on node-based grids, with omega-Jacobi or omega red-black Gauss-Seidel
smoothing, full-weighting restriction, bi-/trilinear interpolation and the
rediscretised coarse operator. It is independent of the grid code in
mg_oracle.c: every operator is replaced by its Fourier symbol.

Two forms are provided:

* ``two_grid_discrete`` works in the sine basis of a Dirichlet grid with
  h = 1/N. The sine modes split into groups of at most 2**dim coupled modes
  (the coarsening harmonics k -> N-k per dimension; the red-black pattern
  couples k with N-k in every dimension at once, which stays in the group),
  so the spectral radius of the full two-grid matrix is the largest spectral
  radius of the group blocks. This is exact for the finite grid.
* ``two_grid_lfa`` / ``smoothing_factor`` are the classical infinite-grid
  suprema over continuous frequencies.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

RBGS = 0
JACOBI = 1


def _c(c, dim):
    return np.array([1.0] * dim if c is None else list(c)[:dim], dtype=np.float64)


def _lam(theta, c, h):
    """Symbol of A: h^-2 sum_d c_d (2 - 2 cos theta_d)."""
    return float(np.sum(c * (2.0 - 2.0 * np.cos(theta)))) / (h * h)


def _smoother_block(thetas, partner, sign, c, h, smoother, omega):
    """Smoother matrix on a set of modes.

    thetas: list of frequency vectors; partner[i]: index of the mode that the
    red-black pattern maps mode i to; sign: the factor chi * phi_i =
    sign * phi_partner[i].
    """
    m = len(thetas)
    D = 2.0 * float(np.sum(c)) / (h * h)
    K = np.diag([1.0 - omega * _lam(t, c, h) / D for t in thetas])
    if smoother == JACOBI:
        return K
    X = np.zeros((m, m))
    for i in range(m):
        X[partner[i], i] += sign
    I = np.eye(m)
    Mr = 0.5 * (I + X)   # projection on red nodes (i+j[+k] even)
    Mb = 0.5 * (I - X)   # projection on black nodes
    S_red = Mb + Mr @ K
    S_black = Mr + Mb @ K
    return S_black @ S_red


def two_grid_discrete(dim, n, smoother, omega, nu1, nu2, c=None):
    """Spectral radius of the two-grid operator on a Dirichlet grid with n nodes per dimension.

    Uses the sine basis phi_k(x) = prod_d sin(k_d pi x_d), k_d in 1..N-1,
    N = n - 1. Per dimension, full weighting maps phi_k (k < N/2) and
    phi_{N-k} to the coarse mode psi_k with factors (1 + cos k pi h)/2 and
    -(1 - cos k pi h)/2, bilinear interpolation maps psi_k back with the same
    factors, and phi_{N/2} has no coarse image. The red-black pattern
    (-1)^(i+j[+k]) maps phi_k to (-1)^dim phi_{N-k}.
    """
    N = n - 1
    if N < 4 or N % 2:
        raise ValueError("n must be 2**m + 1 with m >= 2")
    h = 1.0 / N
    H = 2.0 * h
    c = _c(c, dim)
    sign = (-1.0) ** dim
    rho = 0.0
    for k in itertools.product(range(1, N // 2 + 1), repeat=dim):
        per_dim = [[k[d]] if k[d] == N // 2 else [k[d], N - k[d]] for d in range(dim)]
        modes = list(itertools.product(*per_dim))
        index = {m: i for i, m in enumerate(modes)}
        thetas = [np.array(m, dtype=np.float64) * math.pi * h for m in modes]
        partner = [index[tuple(N - x for x in m)] for m in modes]
        S = _smoother_block(thetas, partner, sign, c, h, smoother, omega)
        msz = len(modes)
        C = np.eye(msz)
        if all(k[d] < N // 2 for d in range(dim)):
            r = np.ones(msz)
            for i, m in enumerate(modes):
                for d in range(dim):
                    ck = math.cos(k[d] * math.pi * h)
                    r[i] *= 0.5 * (1.0 + ck) if m[d] == k[d] else -0.5 * (1.0 - ck)
            lam = np.array([_lam(t, c, h) for t in thetas])
            lamH = float(np.sum(c * (2.0 - 2.0 * np.cos(np.array(k) * math.pi * H)))) / (H * H)
            C = C - np.outer(r, r * lam) / lamH
        M = np.linalg.matrix_power(S, nu2) @ C @ np.linalg.matrix_power(S, nu1)
        rho = max(rho, float(np.max(np.abs(np.linalg.eigvals(M)))))
    return rho


def _harmonics(theta):
    """The 2**dim coarsening harmonics of a low frequency theta in [-pi/2, pi/2)^dim."""
    dim = len(theta)
    out = []
    for alpha in itertools.product((0, 1), repeat=dim):
        t = np.array([theta[d] if alpha[d] == 0 else theta[d] - math.copysign(math.pi, theta[d])
                      for d in range(dim)])
        out.append((alpha, t))
    return out


def _two_grid_symbol(theta, c, smoother, omega, nu1, nu2):
    dim = len(theta)
    h = 1.0
    harm = _harmonics(theta)
    alphas = [a for a, _ in harm]
    thetas = [t for _, t in harm]
    index = {a: i for i, a in enumerate(alphas)}
    partner = [index[tuple(1 - x for x in a)] for a in alphas]
    S = _smoother_block(thetas, partner, 1.0, c, h, smoother, omega)
    r = np.array([float(np.prod((1.0 + np.cos(t)) / 2.0)) for t in thetas])
    lam = np.array([_lam(t, c, h) for t in thetas])
    lamH = float(np.sum(c * (2.0 - 2.0 * np.cos(2.0 * theta)))) / 4.0
    C = np.eye(len(thetas)) - np.outer(r, r * lam) / lamH
    return np.linalg.matrix_power(S, nu2) @ C @ np.linalg.matrix_power(S, nu1), S


def two_grid_lfa(dim, smoother, omega, nu1, nu2, c=None, m=64):
    """Infinite-grid LFA two-grid factor: sup over low frequencies theta != 0,
    sampled on an m**dim grid of [-pi/2, pi/2)^dim shifted off theta = 0."""
    c = _c(c, dim)
    pts = -math.pi / 2 + (np.arange(m) + 0.5) * (math.pi / m)
    rho = 0.0
    for theta in itertools.product(pts, repeat=dim):
        M, _ = _two_grid_symbol(np.array(theta), c, smoother, omega, nu1, nu2)
        rho = max(rho, float(np.max(np.abs(np.linalg.eigvals(M)))))
    return rho


def smoothing_factor(dim, omega, c=None, m=64):
    """omega-Jacobi smoothing factor: sup over high frequencies of |S(theta)|,
    S(theta) = 1 - omega * A(theta) / diag. The frequency grid includes the
    endpoints +-pi/2 and +-pi, where the supremum is attained."""
    c = _c(c, dim)
    pts = np.linspace(-math.pi, math.pi, 2 * m + 1)
    D = 2.0 * float(np.sum(c))
    mu = 0.0
    for theta in itertools.product(pts, repeat=dim):
        t = np.array(theta)
        if np.all(np.abs(t) < math.pi / 2):
            continue  # low frequency
        mu = max(mu, abs(1.0 - omega * _lam(t, c, 1.0) / D))
    return mu
