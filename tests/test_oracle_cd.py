"""Pins of the complex-diffusion oracle (oracle/cd_oracle.c) against facts
fixed by the mathematics (Sec. 4: u_t = div(g(Im u) grad u), Neumann
boundaries, g(s) = e^{i theta} / (1 + (s / (kappa theta))^2), averaged finite
differences in space, implicit Euler in time; cell-centred multigrid with
cell-centred restriction and constant interpolation).

- Diffusivity: g = e^{i theta} where Im u = 0, e^{i theta} / 2 where
  Im u = kappa theta, modulus falling with |Im u|.
- Face coefficients: hand-computed means of the cell values; coarse faces:
  hand-computed means of the two fine faces they span.
- Operator: with Im u^n = 0 the faces are the constant e^{i theta}, and the
  cell-centred Neumann cosine modes are eigenvectors of A with eigenvalue
  1 + tau e^{i theta} sum_d (4/h^2) sin^2(k_d pi h / 2).
- Conservation: sum_p (A u)_p = sum_p u_p for any complex faces (every
  interior flux enters two cells with opposite signs; boundary faces carry
  none), so a time step conserves the mean.
- Red-black Gauss-Seidel with omega = 1 leaves a zero residual on the colour
  updated last; one Jacobi sweep from zero is omega f / diag.
- A time step from a real cosine mode returns the mode divided by its
  eigenvalue; V(2,2) cycles contract by <= 0.15 on a random image.
- With unit faces the operator is tau times the cell-centred oracle's with
  sigma = 1/tau, and the smoothers' iterates agree (two separate sources).
- For the lagged (linear) system one FAS two-grid cycle equals the
  correction scheme's cycle.
"""
import math

import numpy as np
import pytest

import oracle


def rand_c(n, seed, scale_im=1.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, (n, n)) + 1j * scale_im * rng.uniform(-1, 1, (n, n))


def cos_mode(n, kx, ky):
    x = (np.arange(n) + 0.5) / n
    return np.outer(np.cos(ky * math.pi * x), np.cos(kx * math.pi * x))  # rows y, columns x


def test_diffusivity_closed_forms():
    theta, kappa = 0.07, 0.3
    u = np.array([[0.0 + 0.0j, 2.0 + kappa * theta * 1j], [1.0 - kappa * theta * 1j, 5.0 + 0.5j]])
    g = oracle.cd_diffusivity(u, theta, kappa)
    e = np.exp(1j * theta)
    assert abs(g[0, 0] - e) < 1e-15
    assert abs(g[0, 1] - e / 2) < 1e-15 and abs(g[1, 0] - e / 2) < 1e-15
    assert abs(g[1, 1]) < abs(g[0, 1]) and np.allclose(np.angle(g), theta)


def test_faces_and_their_coarsening_by_hand():
    g = np.arange(16).reshape(4, 4) * (1 + 0.5j)
    gx, gy = oracle.cd_faces(g)
    assert gx[2, 1] == 0.5 * (g[2, 1] + g[2, 2]) and gy[1, 3] == 0.5 * (g[1, 3] + g[2, 3])
    assert np.all(gx[:, 3] == 0) and np.all(gy[3, :] == 0)
    cx, cy = oracle.cd_coarsen_faces(gx, gy)
    # coarse x-face between coarse cells (0, J) and (1, J): fine faces at x index 1, rows 2J, 2J+1
    assert cx[1, 0] == 0.5 * (gx[2, 1] + gx[3, 1])
    # coarse y-face between coarse cells (I, 0) and (I, 1): fine faces at row 1, columns 2I, 2I+1
    assert cy[0, 1] == 0.5 * (gy[1, 2] + gy[1, 3])
    assert np.all(cx[:, 1] == 0) and np.all(cy[1, :] == 0)


@pytest.mark.parametrize("n", [8, 32])
def test_constant_faces_have_the_neumann_cosine_modes(n):
    theta, tau = 0.05, 3e-3
    g = np.full((n, n), np.exp(1j * theta))
    gx, gy = oracle.cd_faces(g)
    h = 1.0 / n
    for kx, ky in [(0, 0), (1, 0), (2, 3), (n - 1, 1), (n - 1, n - 1)]:
        u = cos_mode(n, kx, ky)
        lam = 1 + tau * np.exp(1j * theta) * sum(4 / h ** 2 * math.sin(k * math.pi * h / 2) ** 2 for k in (kx, ky))
        Au = oracle.cd_apply(u, tau, gx, gy)
        assert np.max(np.abs(Au - lam * u)) <= 1e-12 * abs(lam), (kx, ky)


def test_conservation_for_any_faces():
    n = 16
    u = rand_c(n, 1)
    g = rand_c(n, 2) + 2.0
    gx, gy = oracle.cd_faces(g)
    Au = oracle.cd_apply(u, 0.01, gx, gy)
    assert abs(Au.sum() - u.sum()) <= 1e-11 * np.abs(Au).sum()


def test_rbgs_zeroes_the_last_colour_and_jacobi_step():
    n, tau = 16, 5e-3
    g = oracle.cd_diffusivity(rand_c(n, 3, 0.01), 0.05, 0.1)
    gx, gy = oracle.cd_faces(g)
    u0, f = rand_c(n, 4), rand_c(n, 5)
    u1 = oracle.cd_smooth(u0, f, tau, gx, gy, 1, smoother=oracle.RBGS, omega=1.0)
    r = oracle.cd_residual(u1, f, tau, gx, gy)
    par = np.add.outer(np.arange(n), np.arange(n)) % 2
    scale = np.max(np.abs(oracle.cd_apply(u1, tau, gx, gy))) + np.max(np.abs(f))
    assert np.max(np.abs(r[par == 1])) <= 1e-13 * scale
    assert np.max(np.abs(r[par == 0])) > 1e-6 * scale
    # Jacobi from zero: omega f / diag, diag read off A applied to a unit vector
    uj = oracle.cd_smooth(np.zeros((n, n), complex), f, tau, gx, gy, 1, smoother=oracle.JACOBI, omega=0.8)
    e = np.zeros((n, n), complex)
    e[0, 5] = 1.0
    d = oracle.cd_apply(e, tau, gx, gy)[0, 5]
    assert abs(uj[0, 5] - 0.8 * f[0, 5] / d) <= 1e-15 * abs(uj[0, 5])


def test_transfers():
    e = rand_c(8, 6)
    fine = oracle.cd_prolong_add(e, np.zeros((16, 16), complex))
    assert np.array_equal(fine[::2, ::2], e) and np.array_equal(fine[1::2, 1::2], e)
    assert np.max(np.abs(oracle.cd_restrict(fine) - e)) <= 4 * np.finfo(float).eps * np.max(np.abs(e))
    r = np.arange(16.0).reshape(4, 4) * (1 - 1j)
    assert np.array_equal(oracle.cd_restrict(r), np.array([[2.5, 4.5], [10.5, 12.5]]) * (1 - 1j))


def test_time_step_of_a_cosine_mode_and_contraction():
    n, theta, kappa, tau = 64, 0.05, 0.1, 2e-3
    u0 = cos_mode(n, 3, 2) + 0j  # real: the lagged diffusivity is e^{i theta} everywhere
    H = oracle.CDHierarchy(n, tau, theta, kappa, smoother=oracle.RBGS, nu1=2, nu2=2)
    assert H.levels == 7
    u1, rho = H.time_step(u0, 1e-13, 30)
    h = 1.0 / n
    lam = 1 + tau * np.exp(1j * theta) * sum(4 / h ** 2 * math.sin(k * math.pi * h / 2) ** 2 for k in (3, 2))
    assert np.max(np.abs(u1 - u0 / lam)) <= 1e-12
    # a random image with a small imaginary part: V(2,2) contracts fast and the
    # step conserves the mean
    img = rand_c(n, 7, 0.02) + 1.0
    u1, rho = H.time_step(img, 1e-12, 30)
    q = (rho[-1] / rho[-4]) ** (1 / 3)
    assert q <= 0.15, rho
    assert abs(u1.sum() - img.sum()) <= 1e-9 * np.abs(img).sum()


def test_real_unit_faces_reduce_to_the_cell_centred_oracle():
    # With every face coefficient 1, A = I + tau L (L the Neumann cell
    # Laplacian), i.e. tau times the cell-centred operator with sigma = 1/tau:
    # two independent oracle sources must agree on the operator and on the
    # smoothers' iterates for the correspondingly scaled right-hand side.
    n, tau = 16, 3e-3
    ones = np.ones((n, n), complex)
    ones[:, -1] = 0.0
    gx = ones.copy()
    gy = np.ones((n, n), complex)
    gy[-1, :] = 0.0
    u = np.random.default_rng(8).uniform(-1, 1, (n, n))
    f = np.random.default_rng(9).uniform(-1, 1, (n, n))
    Au_cd = oracle.cd_apply(u + 0j, tau, gx, gy)
    Au_cc = oracle.cc_apply(u, sigma=1.0 / tau, bc="neumann")
    assert np.max(np.abs(Au_cd - tau * Au_cc)) <= 1e-12 * np.max(np.abs(Au_cd))
    for sm, om in ((oracle.RBGS, 1.0), (oracle.JACOBI, 0.8)):
        a = oracle.cd_smooth(u + 0j, f + 0j, tau, gx, gy, 3, smoother=sm, omega=om)
        b = oracle.cc_smooth(u, f / tau, 3, smoother=sm, omega=om, sigma=1.0 / tau, bc="neumann")
        assert np.max(np.abs(a.imag)) == 0.0
        assert np.max(np.abs(a.real - b)) <= 1e-12 * np.max(np.abs(b)), sm


def test_fas_and_correction_scheme_coincide_for_the_lagged_system():
    # With the diffusivity lagged, a step's system is linear; one FAS two-grid
    # cycle (coarse problem A_H v = A_H(R u) + R(f - A u), correction
    # u += P(v - R u)) then equals the correction scheme's cycle (A_H e = R r,
    # u += P e) up to rounding, which is why the correction scheme is used.
    n, tau = 16, 4e-3
    g = oracle.cd_diffusivity(rand_c(n, 10, 0.02), 0.05, 0.1)
    gx, gy = oracle.cd_faces(g)
    cx, cy = oracle.cd_coarsen_faces(gx, gy)
    nc = n // 2

    def coarse_solve(rhs):
        cols = []
        for k in range(nc * nc):
            e = np.zeros(nc * nc, complex)
            e[k] = 1.0
            cols.append(oracle.cd_apply(e.reshape(nc, nc), tau, cx, cy).reshape(-1))
        return np.linalg.solve(np.array(cols).T, rhs.reshape(-1)).reshape(nc, nc)

    f = rand_c(n, 11)
    u0 = oracle.cd_smooth(rand_c(n, 12), f, tau, gx, gy, 2)
    r = oracle.cd_residual(u0, f, tau, gx, gy)
    # correction scheme
    u_cs = oracle.cd_prolong_add(coarse_solve(oracle.cd_restrict(r)), u0)
    # full approximation scheme
    Ru = oracle.cd_restrict(u0)
    v = coarse_solve(oracle.cd_apply(Ru, tau, cx, cy) + oracle.cd_restrict(r))
    u_fas = oracle.cd_prolong_add(v - Ru, u0)
    assert np.max(np.abs(u_fas - u_cs)) <= 1e-12 * np.max(np.abs(u_cs))


def test_norms_closed_form():
    # |3 + 4i| = 5 in every one of n^2 cells: the norm is 5 n; likewise the
    # cell-centred oracle's norm of a constant field
    n = 16
    assert oracle.cd_norm(np.full((n, n), 3 + 4j)) == 5.0 * n
    assert oracle.cc_norm(np.full((n, n), -2.0)) == 2.0 * n
    assert oracle.cc_norm(np.full((8, 8, 8), 0.5)) == 0.5 * math.sqrt(512)
