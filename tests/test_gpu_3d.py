"""Parity of the plane-marching 3D kernels (constant 7-point stencil) with
the oracle at sizes where a level spans several x-tiles (64 FP64, 128 FP32 or
256 BF16 columns per tile), several y-tiles with a ragged last one (8 rows per
block, n - 2 interior rows) and several z-chunks, and at the full 513^3
workload in the launch configuration bench.py times."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import OP_TOL, error_vs_converged_oracle, interior, need_gpu, rel_err, zero_boundary

pytestmark = pytest.mark.gpu


def solver(prec, n, smoother="jacobi", omega=6 / 7, nu=(2, 2), maxit=60, **kw):
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    return Solver(3, n, precision=prec, smoother=smoother, omega=omega, nu1=nu[0], nu2=nu[1], maxit=maxit, **kw)


def upload(s, level, field, a):
    s.set_field(level, field, a)
    return s.get_field(level, field)


@pytest.mark.parametrize("prec,n", [("fp64", 129), ("fp32_dc", 257), ("bf16_dc", 513)])
def test_level0_operators_multi_tile(prec, n):
    s = solver(prec, n)
    tol = OP_TOL[prec]
    nc = s.level_size(1)
    u = upload(s, 0, "u", zero_boundary(synth.uniform(11, (n,) * 3)))
    f = upload(s, 0, "f", synth.uniform(12, (n,) * 3))
    # residual
    s.residual(0)
    r = s.get_field(0, "r")
    assert rel_err(interior(r), interior(oracle.residual(u, f))) <= tol
    # full weighting of that residual into level 1
    r = upload(s, 0, "r", r)
    s.restrict(0)
    fc = s.get_field(1, "f")
    assert rel_err(interior(fc), interior(oracle.restrict(r))) <= tol
    # trilinear interpolation and correction from level 1
    ec = upload(s, 1, "u", zero_boundary(synth.uniform(13, (nc,) * 3)))
    u = upload(s, 0, "u", zero_boundary(synth.uniform(14, (n,) * 3)))
    s.prolongate(0)
    got = s.get_field(0, "u")
    want = oracle.prolong_add(ec, u)
    assert rel_err(interior(got), interior(want)) <= tol
    # one omega-Jacobi sweep
    u = upload(s, 0, "u", zero_boundary(synth.uniform(15, (n,) * 3)))
    s.smooth(0, 1)
    got = s.get_field(0, "u")
    want = oracle.jacobi(u, f, sweeps=1, omega=6 / 7)
    assert rel_err(interior(got), interior(want)) <= 2 * tol


@pytest.mark.parametrize("prec,n", [("fp64", 129), ("fp32_dc", 257)])
def test_rbgs_sweeps_multi_tile(prec, n):
    s = solver(prec, n, smoother="rbgs", omega=1.1, nu=(2, 1))
    u = upload(s, 0, "u", zero_boundary(synth.uniform(21, (n,) * 3)))
    f = upload(s, 0, "f", synth.uniform(22, (n,) * 3))
    s.smooth(0, 2)
    got = s.get_field(0, "u")
    want = oracle.rbgs(u, f, sweeps=2, omega=1.1)
    assert rel_err(interior(got), interior(want)) <= 4 * OP_TOL[prec]


@pytest.mark.parametrize("smoother,omega,nu", [("jacobi", 6 / 7, (2, 2)), ("rbgs", 1.0, (2, 1))])
def test_fp64_cycles_match_oracle_129(smoother, omega, nu):
    n = 129
    f = synth.normal_rhs(3, n, 0x5EED0003)
    s = solver("fp64", n, smoother=smoother, omega=omega, nu=nu, maxit=3)
    s.set_rhs(f)
    _, _, hist = s.solve(0.0, raise_on_noconv=False)
    ref = oracle.Hierarchy(3, n, smoother=0 if smoother == "rbgs" else 1, omega=omega, nu1=nu[0], nu2=nu[1])
    ref.set_rhs(f)
    rho = ref.solve(0.0, 3)
    assert np.max(np.abs(hist - rho)) <= 1e-12, (hist, rho)
    assert rel_err(s.get_solution(), ref.get_u()) <= 1e-11


def test_fp32_dc_257_reaches_tolerance():
    n = 257
    f = synth.normal_rhs(3, n, 0x5EED0003)
    s = solver("fp32_dc", n, inner_cycles=2)
    s.set_rhs(f)
    it, rr, _ = s.solve(1e-10)
    assert rr <= 1e-10
    u = s.get_solution()
    rel = oracle.norm(oracle.residual(u, f)) / oracle.norm(f)
    assert rel <= 1.01e-10, rel


def test_fullsize_config3_bf16_dc_reaches_tolerance():
    # 513^3, f ~ N(0,1) (seed 0x5EED0003), Jacobi omega = 6/7 V(2,2), BF16-stored
    # inner cycles in FP64 defect correction: the oracle recomputes the FP64
    # residual of the GPU's answer over the whole grid.
    n = 513
    f = synth.normal_rhs(3, n, 0x5EED0003)
    s = solver("bf16_dc", n, inner_cycles=2)
    s.set_rhs(f)
    it, rr, _ = s.solve(1e-10)
    assert rr <= 1e-10
    u = s.get_solution()
    del s
    rel = oracle.norm(oracle.residual(u, f, mt=True), mt=True) / oracle.norm(f, mt=True)
    assert rel <= 1.01e-10, rel
    # final error against the oracle's FP64 solution converged from zero,
    # within the guaranteed bound (residuals of both over lambda_min(A))
    err, bound, orr = error_vs_converged_oracle(u, f, maxit=40, smoother=oracle.JACOBI, omega=6.0 / 7.0,
                                                nu1=2, nu2=2)
    print(f"513^3 BF16-DC: rel l2 error vs oracle {err:.3e} (bound {bound:.3e}, oracle relres {orr:.2e})")
    assert orr <= 1e-12
    assert err <= bound, (err, bound)
