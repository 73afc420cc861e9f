"""Pins of the cell-centred oracle (oracle/cc_oracle.c) against facts fixed by
the mathematics, not by re-typing its formulas.

Grid: n = 2^m cells per dimension, h = 1/n, centres x_i = (i + 1/2) h.
Operator: sigma u - sum_d c_d d^2/dx_d^2 by finite volumes, with Neumann
(zero flux) or homogeneous Dirichlet (ghost -u_p) boundary faces (Table 1:
cell-centred grids, Neumann/Dirichlet boundaries; Sec. 4).

- Spectrum: the discrete Neumann operator has the eigenvectors
  prod_d cos(k_d pi x_d) and the Dirichlet one prod_d sin(k_d pi x_d), with
  eigenvalue sigma + sum_d c_d (4/h^2) sin^2(k_d pi h / 2). A wrong boundary
  term, a dropped coefficient or a wrong h breaks it.
- Symmetry <v, A u> = <A v, u>, and for Neumann faces the conservation
  sum_p (A u)_p = sigma sum_p u_p (interior fluxes cancel, boundary fluxes
  vanish).
- Red-black Gauss-Seidel with omega = 1 leaves a zero residual on the cells
  of the colour it updated last (each black cell is solved exactly against
  red neighbours that no longer change); this pins the diagonal and the
  colouring.
- Restriction of a hand-computed 4x4 example; restriction of a constant
  interpolation returns the coarse field (up to the rounding of the sum).
- The dense solve satisfies A u = f with the pinned operator.
- The V-cycle converges to the discrete solution, whose error against the
  manufactured solutions cos(pi x) cos(pi y) (Neumann) and sin(pi x) sin(pi y)
  (Dirichlet) falls as O(h^2); V(2,1) RBGS contracts by a factor <= 0.3 per
  cycle, and a single-level hierarchy is the dense solve.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def centres(n):
    return (np.arange(n) + 0.5) / n


def mode(dim, n, ks, bc):
    x = centres(n)
    fn = np.cos if bc == "neumann" else np.sin
    out = np.ones((n,) * dim)
    for d, k in enumerate(ks):  # axis d varies along numpy axis dim-1-d (x fastest)
        shape = [1] * dim
        shape[dim - 1 - d] = n
        out = out * fn(k * math.pi * x).reshape(shape)
    return out


@pytest.mark.parametrize("dim,n", [(2, 8), (2, 16), (3, 8)])
@pytest.mark.parametrize("bc", ["neumann", "dirichlet"])
def test_eigenvectors(dim, n, bc):
    c = (1.0, 2.5, 0.5)[:dim]
    sigma = 3.0
    h = 1.0 / n
    rng = np.random.default_rng(1)
    for _ in range(6):
        lo = 0 if bc == "neumann" else 1
        ks = [int(rng.integers(lo, n)) if bc == "neumann" else int(rng.integers(1, n + 1)) for _ in range(dim)]
        u = mode(dim, n, ks, bc)
        lam = sigma + sum(cd * 4.0 / h ** 2 * math.sin(k * math.pi * h / 2) ** 2 for cd, k in zip(c, ks))
        Au = oracle.cc_apply(u, c=c, sigma=sigma, bc=bc)
        assert np.max(np.abs(Au - lam * u)) <= 1e-12 * lam * max(1.0, np.max(np.abs(u))), (ks, bc)


@pytest.mark.parametrize("dim,n", [(2, 16), (3, 8)])
@pytest.mark.parametrize("bc", ["neumann", "dirichlet"])
def test_symmetry_and_conservation(dim, n, bc):
    u = synth.uniform(3, (n,) * dim) - 0.5
    v = synth.uniform(4, (n,) * dim) - 0.5
    c, sigma = (1.0, 0.7, 1.9)[:dim], 0.25
    Au = oracle.cc_apply(u, c=c, sigma=sigma, bc=bc)
    Av = oracle.cc_apply(v, c=c, sigma=sigma, bc=bc)
    assert abs(np.sum(v * Au) - np.sum(Av * u)) <= 1e-11 * np.sum(np.abs(v * Au))
    if bc == "neumann":
        assert abs(np.sum(Au) - sigma * np.sum(u)) <= 1e-10 * np.sum(np.abs(Au))


@pytest.mark.parametrize("dim,n", [(2, 16), (3, 8)])
@pytest.mark.parametrize("bc", ["neumann", "dirichlet"])
def test_rbgs_zeroes_the_last_colour(dim, n, bc):
    u0 = synth.uniform(5, (n,) * dim)
    f = synth.uniform(6, (n,) * dim) - 0.5
    kw = dict(c=(1.0, 3.0, 0.5)[:dim], sigma=0.5, bc=bc)
    u1 = oracle.cc_smooth(u0, f, 1, smoother=oracle.RBGS, omega=1.0, **kw)
    r = oracle.cc_residual(u1, f, **kw)
    par = sum(np.indices((n,) * dim)) % 2
    scale = np.max(np.abs(oracle.cc_apply(u1, **kw))) + np.max(np.abs(f))
    assert np.max(np.abs(r[par == 1])) <= 1e-13 * scale
    assert np.max(np.abs(r[par == 0])) > 1e-6 * scale  # red cells saw black values change


def test_jacobi_is_the_diagonal_step():
    # from u0 = 0 one omega-Jacobi sweep gives omega f / diag; the diagonal is
    # the one pinned by the RBGS test through the residual
    n, dim = 16, 2
    f = synth.uniform(7, (n, n)) - 0.5
    for bc in ("neumann", "dirichlet"):
        d = oracle.cc_diag(dim, n, sigma=0.5, bc=bc)
        u1 = oracle.cc_smooth(np.zeros((n, n)), f, 1, smoother=oracle.JACOBI, omega=0.8, sigma=0.5, bc=bc)
        assert np.allclose(u1, 0.8 * f / d, rtol=1e-15, atol=0)
        # and diag is the response of A at a cell to a unit value there
        e = np.zeros((n, n))
        e[0, 3] = 1.0
        assert oracle.cc_apply(e, sigma=0.5, bc=bc)[0, 3] == d[0, 3]


def test_restriction_hand_example_and_transfer_identities():
    r = np.arange(16.0).reshape(4, 4)
    want = np.array([[2.5, 4.5], [10.5, 12.5]])  # mean of each 2x2 block
    assert np.array_equal(oracle.cc_restrict(r), want)
    for dim, nc in [(2, 8), (3, 4)]:
        e = synth.uniform(8, (nc,) * dim)
        fine = oracle.cc_prolong_add(e, np.zeros((2 * nc,) * dim))
        # the mean of 2^dim equal values: exact up to the rounding of the sum
        assert np.max(np.abs(oracle.cc_restrict(fine) - e)) <= 4 * np.finfo(float).eps * np.max(np.abs(e))
        assert np.array_equal(fine[(slice(None, None, 2),) * dim], e)
        assert np.array_equal(fine[(slice(1, None, 2),) * dim], e)
        base = synth.uniform(9, (2 * nc,) * dim)
        assert np.array_equal(oracle.cc_prolong_add(e, base) - base, fine)


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 4)])
@pytest.mark.parametrize("bc,sigma", [("neumann", 0.5), ("dirichlet", 0.0)])
def test_dense_solve(dim, n, bc, sigma):
    f = synth.uniform(10, (n,) * dim) - 0.5
    u = oracle.cc_dense_solve(f, sigma=sigma, bc=bc)
    r = f - oracle.cc_apply(u, sigma=sigma, bc=bc)
    assert np.max(np.abs(r)) <= 1e-12 * np.max(np.abs(f))


@pytest.mark.parametrize("bc", ["neumann", "dirichlet"])
def test_manufactured_solution_second_order(bc):
    sigma = 1.0
    errs = []
    for n in (16, 32, 64, 128):
        ustar = mode(2, n, (1, 1), bc)
        f = (sigma + 2 * math.pi ** 2) * ustar
        H = oracle.CCHierarchy(2, n, sigma=sigma, bc=bc)
        H.set_rhs(f)
        rho = H.solve(1e-11, 40)
        assert rho[-1] <= 1e-11
        errs.append(np.max(np.abs(H.get_u() - ustar)))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.6 < q < 4.4 for q in ratios), (errs, ratios)


@pytest.mark.parametrize("dim,n", [(2, 128), (3, 32)])
@pytest.mark.parametrize("bc,sigma", [("neumann", 1.0), ("dirichlet", 0.0)])
def test_vcycle_contraction(dim, n, bc, sigma):
    f = synth.uniform(11, (n,) * dim) - 0.5
    H = oracle.CCHierarchy(dim, n, sigma=sigma, bc=bc, smoother=oracle.RBGS, nu1=2, nu2=1)
    assert H.levels == int(math.log2(n)) + 1
    H.set_rhs(f)
    rho = H.solve(0.0, 10)
    q = (rho[10] / rho[5]) ** (1 / 5)
    assert q <= 0.3, rho


def test_single_level_hierarchy_is_the_dense_solve():
    f = synth.uniform(12, (8, 8)) - 0.5
    H = oracle.CCHierarchy(2, 8, sigma=2.0, bc="neumann", coarsest_n=8)
    assert H.levels == 1
    H.set_rhs(f)
    H.vcycle()
    assert np.array_equal(H.get_u(), oracle.cc_dense_solve(f, sigma=2.0, bc="neumann"))
