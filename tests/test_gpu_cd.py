"""Complex diffusion (include/mg_cd.h) against the complex-diffusion oracle.

A step's coefficients (cell diffusivity from Im u^n, averaged faces, the
coarse faces of every level), every level operator on seeded complex fields
with those faces (complex red-black Gauss-Seidel and Jacobi, residual,
restriction, constant interpolation) and whole time steps (V-cycle history
to 1e-12 per cycle, the new state to 1e-11) must match the oracle; a real
cosine image must come out divided by its closed-form eigenvalue, and a step
conserves the mean (Neumann faces carry no flux) up to the sum of its final
residual.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_util import need_gpu, rel_err

pytestmark = pytest.mark.gpu

THETA, KAPPA = math.pi / 30, 0.1


def image(n, seed, im=0.02):
    rng = np.random.default_rng(seed)
    # a smooth bump plus noise: the kind of image Sec. 4 denoises
    x = (np.arange(n) + 0.5) / n
    base = np.exp(-((x[None, :] - 0.5) ** 2 + (x[:, None] - 0.4) ** 2) / 0.05)
    return base + 0.3 * rng.uniform(-1, 1, (n, n)) + 1j * im * rng.uniform(-1, 1, (n, n))


def conserved(s, u0, u1):
    # sum(A u) = sum(u) exactly, so sum(u1) - sum(u0) = -sum(r) for the final
    # residual r = u0 - A u1, and |sum(r)| <= sqrt(N) ||r||
    bound = math.sqrt(u0.size) * s.residual_norm() + 1e-12 * np.abs(u0).sum()
    assert abs(u1.sum() - u0.sum()) <= bound, (abs(u1.sum() - u0.sum()), bound)


def make(n, tau, **kw):
    need_gpu()
    from paper_1406_5369_gb300 import CDSolver
    return CDSolver(n, tau=tau, theta=THETA, kappa=KAPPA, **kw)


@pytest.mark.parametrize("n", [256, 128])
def test_step_coefficients_every_level(n):
    tau = 1e-3
    s = make(n, tau)
    ref = oracle.CDHierarchy(n, tau, THETA, KAPPA)
    u0 = image(n, 1)
    s.begin_step(u0)
    ref.begin_step(u0)
    assert s.levels == ref.levels
    for l in range(s.levels):
        gx, gy = ref.faces(l)
        assert rel_err(s.get_field(l, "gx"), gx) <= 1e-14, l
        assert rel_err(s.get_field(l, "gy"), gy) <= 1e-14, l
    assert np.array_equal(s.get_field(0, "f"), u0) and np.array_equal(s.get_field(0, "u"), u0)


@pytest.mark.parametrize("smoother,omega", [("rbgs", 1.0), ("jacobi", 0.8)])
def test_level_operators(smoother, omega):
    n, tau = 256, 4e-3
    s = make(n, tau, smoother=smoother, omega=omega)
    ref = oracle.CDHierarchy(n, tau, THETA, KAPPA)
    u0 = image(n, 2, im=0.05)
    s.begin_step(u0)
    ref.begin_step(u0)
    sm = oracle.RBGS if smoother == "rbgs" else oracle.JACOBI
    rng = np.random.default_rng(3)
    for l in range(s.levels):
        nl = s.level_size(l)
        gx, gy = ref.faces(l)
        u = rng.uniform(-1, 1, (nl, nl)) + 1j * rng.uniform(-1, 1, (nl, nl))
        f = rng.uniform(-1, 1, (nl, nl)) + 1j * rng.uniform(-1, 1, (nl, nl))
        s.set_field(l, "u", u)
        s.set_field(l, "f", f)
        s.smooth(l, 2)
        want = oracle.cd_smooth(u, f, tau, gx, gy, 2, smoother=sm, omega=omega)
        assert rel_err(s.get_field(l, "u"), want) <= 1e-13, (l, nl)
        s.set_field(l, "u", u)
        s.residual(l)
        r = s.get_field(l, "r")
        assert rel_err(r, oracle.cd_residual(u, f, tau, gx, gy)) <= 1e-13, (l, nl)
        if l + 1 < s.levels:
            s.restrict(l)
            assert rel_err(s.get_field(l + 1, "f"), oracle.cd_restrict(r)) <= 1e-15, (l, nl)
            e = rng.uniform(-1, 1, (nl // 2, nl // 2)) + 0j
            s.set_field(l + 1, "u", e)
            s.prolongate(l)
            assert np.array_equal(s.get_field(l, "u"), oracle.cd_prolong_add(e, u)), (l, nl)


@pytest.mark.parametrize("n,tau,smoother,omega,nu", [(256, 1e-3, "rbgs", 1.0, (2, 2)), (512, 1e-2, "jacobi", 0.8, (2, 2)),
                                                     (128, 1e-1, "rbgs", 1.0, (1, 1))])
def test_time_step_matches_oracle(n, tau, smoother, omega, nu):
    cycles = 8
    s = make(n, tau, smoother=smoother, omega=omega, nu1=nu[0], nu2=nu[1], maxit=cycles)
    ref = oracle.CDHierarchy(n, tau, THETA, KAPPA, smoother=oracle.RBGS if smoother == "rbgs" else oracle.JACOBI,
                             omega=omega, nu1=nu[0], nu2=nu[1])
    u0 = image(n, 4)
    _, _, hist = s.time_step(u0, 0.0, raise_on_noconv=False)
    u1_ref, rho = ref.time_step(u0, 0.0, cycles)
    assert len(hist) == len(rho)
    assert np.max(np.abs(hist - rho) / np.maximum(1.0, rho)) <= 1e-12, (hist, rho)
    u1 = s.get_field(0, "u")
    assert rel_err(u1, u1_ref) <= 1e-11
    conserved(s, u0, u1)


def test_cosine_image_and_repeated_steps():
    n, tau = 512, 2e-4
    x = (np.arange(n) + 0.5) / n
    u0 = np.outer(np.cos(2 * math.pi * x), np.cos(3 * math.pi * x)) + 0j  # real: faces e^{i theta}
    s = make(n, tau, maxit=30)
    it, rr, _ = s.time_step(u0, 1e-12)
    h = 1.0 / n
    lam = 1 + tau * np.exp(1j * THETA) * sum(4 / h ** 2 * math.sin(k * math.pi * h / 2) ** 2 for k in (3, 2))
    assert rel_err(s.get_field(0, "u"), u0 / lam) <= 1e-11
    # three steps of a noisy image: each to 1e-10, mean conserved, noise damped
    u = image(n, 5)
    for _ in range(3):
        s.time_step(u, 1e-10)
        un = s.get_field(0, "u")
        conserved(s, u, un)
        u = un
    assert np.std(np.diff(u.real, axis=1)) < np.std(np.diff(image(n, 5).real, axis=1))
