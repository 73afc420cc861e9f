"""LFA in the product (paper_1406_5369_gb300.lfa) and the autotuner's choice
built on it: the LFA-driven choice of smoother, omega and nu.

Pins: the classical two-grid factors of red-black Gauss-Seidel with full
weighting and bilinear interpolation, 0.250 / 0.074 / 0.053 for nu = 1, 2, 3
in 2D; the closed-form omega-Jacobi smoothing factors 3/5 (2D, omega 4/5) and
5/7 (3D, omega 6/7); agreement with the oracle's independent LFA
(oracle.lfa, a separate implementation) over smoothers, weights, sweep counts,
dimensions and anisotropy; and measured oracle V-cycle factors for the
configuration LFA chooses, which must beat the default omega = 1 as predicted.
For cell-centred grids (mean restriction, constant interpolation) the
prediction is checked against the oracle's two-grid iteration matrix,
assembled column by column on a Neumann grid.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.lfa as olfa
import synth
from paper_1406_5369_gb300 import autotune, lfa


def test_classical_red_black_two_grid_factors():
    for nu, want in ((1, 0.250), (2, 0.074), (3, 0.053)):
        got = lfa.two_grid_factor(2, "rbgs", 1.0, nu, 0)
        assert abs(got - want) < 1.5e-3, (nu, got)


def test_jacobi_smoothing_factor_closed_forms():
    assert abs(lfa.smoothing_factor(2, "jacobi", 0.8) - 3 / 5) < 1e-4
    assert abs(lfa.smoothing_factor(3, "jacobi", 6 / 7) - 5 / 7) < 1e-4


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("smoother,omega,nu", [("rbgs", 1.0, (2, 1)), ("rbgs", 1.2, (1, 1)),
                                               ("jacobi", 0.8, (2, 2)), ("jacobi", 6 / 7, (1, 1))])
@pytest.mark.parametrize("c", [(1.0, 1.0, 1.0), (1.0, 3.0, 1.0)])
def test_agrees_with_the_oracle_lfa(dim, smoother, omega, nu, c):
    a = lfa.two_grid_factor(dim, smoother, omega, nu[0], nu[1], c=c)
    # the oracle samples 64^2 frequencies in 2D; 20^3 in 3D keeps it to seconds
    b = olfa.two_grid_lfa(dim, olfa.RBGS if smoother == "rbgs" else olfa.JACOBI, omega, nu[0], nu[1], c=c,
                          m=64 if dim == 2 else 20)
    # both are suprema over sampled frequencies: the oracle's plain sample is a
    # lower bound of the product's refined one, which may exceed it by the
    # sampling error of the coarser 3D sample
    assert b <= a * (1 + 1e-6) + 1e-9, (a, b)
    assert a <= b * (1.02 if dim == 2 else 1.06) + 1e-4, (a, b)


def test_choice_for_2d_poisson_and_its_measured_factor():
    best = autotune.lfa_choice(2, smoothers=("rbgs",), nus=[(2, 1)])
    assert best["smoother"] == "rbgs" and (best["nu1"], best["nu2"]) == (2, 1)
    assert 1.05 <= best["omega"] <= 1.25 and best["rho"] < 0.03
    default = lfa.two_grid_factor(2, "rbgs", 1.0, 2, 1)
    assert best["rho"] < 0.5 * default
    # the oracle's V-cycle on 129^2 shows the predicted gain
    n = 129
    f = synth.uniform_rhs(2, n, 0x5EED00F3)
    q = {}
    for om in (1.0, best["omega"]):
        H = oracle.Hierarchy(2, n, smoother=oracle.RBGS, omega=om, nu1=2, nu2=1)
        H.set_rhs(f)
        rho = H.solve(0.0, 8)
        q[om] = (rho[8] / rho[3]) ** (1 / 5)
    assert q[best["omega"]] <= 1.3 * best["rho"] + 0.005, q
    assert q[best["omega"]] < 0.6 * q[1.0], q


def test_full_ranking_prefers_red_black_and_costs_are_consistent():
    ranked = autotune.lfa_choice(2)["ranking"]
    assert ranked[0]["smoother"] == "rbgs"
    for r in ranked:
        assert r["cycles"] == max(1, math.ceil(math.log(1e-10) / math.log(r["rho"])))
        assert np.isclose(r["words"], r["cycles"] * lfa.cycle_words(2, r["nu1"], r["nu2"]))
    # V(2,1) in 2D: (3*3 + 3 + 1.25 + 0.25 + 2.25) * 4/3 = 21 words per fine node (operator model)
    assert np.isclose(lfa.cycle_words(2, 2, 1), 21.0)
    assert np.isclose(lfa.cycle_words(3, 2, 2), 21.0)


def _cc_two_grid_matrix(n, smoother, omega, nu1, nu2, sigma=1e-3, dim=2):
    """The oracle's cell-centred two-grid error propagation on an n^dim Neumann
    grid, column by column (smooth, residual, restrict, exact coarse solve,
    interpolate, smooth, all with f = 0)."""
    N = n ** dim
    M = np.zeros((N, N))
    z = np.zeros((n,) * dim)
    kw = dict(sigma=sigma, bc="neumann")
    for k in range(N):
        u = np.zeros(N)
        u[k] = 1.0
        u = u.reshape((n,) * dim)
        if nu1:
            u = oracle.cc_smooth(u, z, nu1, smoother=smoother, omega=omega, **kw)
        ec = oracle.cc_dense_solve(oracle.cc_restrict(oracle.cc_residual(u, z, **kw)), **kw)
        u = oracle.cc_prolong_add(ec, u)
        if nu2:
            u = oracle.cc_smooth(u, z, nu2, smoother=smoother, omega=omega, **kw)
        M[:, k] = u.reshape(-1)
    return M


@pytest.mark.parametrize("smoother,omega,nu,tol", [("jacobi", 0.8, (2, 2), 0.03), ("jacobi", 0.6, (1, 1), 0.03),
                                                   ("rbgs", 1.0, (1, 1), 0.12), ("rbgs", 1.0, (2, 1), 0.35)])
def test_cell_centred_lfa_matches_the_oracle_two_grid_matrix(smoother, omega, nu, tol):
    # Neumann faces with a tiny shift: the cell-centred grid is half of a
    # periodic grid with even symmetry, so the infinite-grid symbols apply up
    # to boundary effects, which grow for red-black at small factors
    M = _cc_two_grid_matrix(16, oracle.RBGS if smoother == "rbgs" else oracle.JACOBI, omega, *nu)
    measured = float(np.max(np.abs(np.linalg.eigvals(M))))
    pred = lfa.cc_two_grid_factor(2, smoother, omega, *nu)
    assert abs(measured - pred) <= tol * pred + 1e-3, (measured, pred)


def test_cell_centred_lfa_in_3d():
    # 8^3 cells: Jacobi omega 6/7 V(1,1) attains its supremum on this grid
    M = _cc_two_grid_matrix(8, oracle.JACOBI, 6 / 7, 1, 1, dim=3)
    measured = float(np.max(np.abs(np.linalg.eigvals(M))))
    pred = lfa.cc_two_grid_factor(3, "jacobi", 6 / 7, 1, 1)
    assert abs(measured - pred) <= 0.03 * pred, (measured, pred)


def test_cell_centred_choice():
    best = autotune.lfa_choice(2, grid="cell")
    assert best["smoother"] == "rbgs" and best["rho"] < 0.1
    # the lower-order transfers cost red-black GS V(1,1) its classical 0.074
    assert lfa.cc_two_grid_factor(2, "rbgs", 1.0, 1, 1) > 1.5 * lfa.two_grid_factor(2, "rbgs", 1.0, 1, 1)
