"""Parity of the fused fine-level kernels (smoothing + residual + restriction,
interpolation + smoothing in one pass) with the oracle and with the
one-kernel-per-operator path, including the full-size workloads in the
launch configuration bench.py times."""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import error_vs_converged_oracle, need_gpu, rel_err

pytestmark = pytest.mark.gpu


def history(dim, n, f, cycles, **kw):
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    u0 = kw.pop("u0", None)
    s = Solver(dim, n, maxit=cycles, **kw)
    s.set_rhs(f)
    if u0 is not None:
        s.set_solution(u0)
    _, _, hist = s.solve(0.0, raise_on_noconv=False)
    return s, hist


def oracle_history(dim, n, f, cycles, c=None, omega=1.0, nu1=2, nu2=1, dirichlet=None, u0=None):
    ref = oracle.Hierarchy(dim, n, c=c, omega=omega, nu1=nu1, nu2=nu2)
    ref.set_rhs(f)
    ub = np.zeros((n,) * dim) if dirichlet is None else dirichlet.copy()
    ub[(slice(1, -1),) * dim] = 0.0 if u0 is None else u0[(slice(1, -1),) * dim]
    ref.set_u(ub)
    return ref, ref.solve(0.0, cycles)


@pytest.mark.parametrize("n", [33, 65, 129, 257, 1025, 2049])
@pytest.mark.parametrize("nu1,nu2,omega", [(2, 1, 1.0), (1, 2, 1.0), (1, 1, 1.2), (2, 2, 0.9)])
def test_fused_fp64_matches_oracle(n, nu1, nu2, omega):
    f = synth.uniform_rhs(2, n, 0x5EED0002 ^ n)
    cycles = 6
    s, hist = history(2, n, f, cycles, nu1=nu1, nu2=nu2, omega=omega)
    ref, rho = oracle_history(2, n, f, cycles, omega=omega, nu1=nu1, nu2=nu2)
    assert np.max(np.abs(hist - rho)) <= 1e-12
    assert rel_err(s.get_solution(), ref.get_u()) <= 1e-11


def test_fused_fp64_dirichlet_initial_guess_anisotropic():
    n = 513
    g = synth.uniform(41, (n, n))
    f = synth.uniform_rhs(2, n, 42)
    u0 = synth.random_u0(2, n, 43)
    c = (1.0, 0.5, 1.0)
    s, hist = history(2, n, f, 5, dirichlet=g, u0=u0, stencil=c)
    ref, rho = oracle_history(2, n, f, 5, c=c, dirichlet=g, u0=u0)
    assert np.max(np.abs(hist - rho)) <= 1e-12
    u = s.get_solution()
    assert np.array_equal(u[-1], g[-1]) and np.array_equal(u[:, 0], g[:, 0])
    assert rel_err(u, ref.get_u()) <= 1e-11


@pytest.mark.parametrize("prec", ["fp64", "fp32_dc"])
def test_fused_equals_unfused(prec):
    n = 1025
    f = synth.uniform_rhs(2, n, 44)
    a, ha = history(2, n, f, 5, precision=prec, fuse=True)
    b, hb = history(2, n, f, 5, precision=prec, fuse=False)
    if prec == "fp64":
        assert np.max(np.abs(ha - hb)) <= 1e-12
    else:  # FP32 inner cycles: the two paths round differently
        assert np.all(np.abs(ha - hb) <= 1e-5 * hb + 1e-12)
    assert rel_err(a.get_solution(), b.get_solution()) <= (1e-11 if prec == "fp64" else 1e-5)


def test_fused_config1_closed_form():
    n = 129
    s, hist = history(2, n, synth.sine_rhs(2, n), 12)
    h = 1.0 / (n - 1)
    ch = (math.pi * h / 2) ** 2 / math.sin(math.pi * h / 2) ** 2
    assert np.max(np.abs(s.get_solution() - ch * synth.sine_solution(2, n))) < 1e-11


# ------------------------------------------------------------ full size

def test_fullsize_config2_fp64_cycles_match_oracle():
    # 8193^2, f ~ U[-1,1] (seed 0x5EED0002), V(2,1) RBGS: the bench workload in
    # the bench's launch configuration (fused kernels, graph replay); the first
    # two cycles' relative residuals against the oracle's.
    n = 8193
    f = synth.uniform_rhs(2, n, 0x5EED0002)
    s, hist = history(2, n, f, 2)
    ref, rho = oracle_history(2, n, f, 2)
    assert np.max(np.abs(hist - rho)) <= 1e-12, (hist, rho)
    u = s.get_solution()
    # sampled rows of the solution after two cycles
    uo = ref.get_u()
    for r in (1, 2, 4095, 4096, 8191):
        assert rel_err(u[r], uo[r]) <= 1e-11


def test_fullsize_config2_fp32_dc_reaches_tolerance():
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    n = 8193
    f = synth.uniform_rhs(2, n, 0x5EED0002)
    s = Solver(2, n, precision="fp32_dc", maxit=40)
    s.set_rhs(f)
    it, rr, hist = s.solve(1e-10)
    assert rr <= 1e-10
    u = s.get_solution()
    # the oracle recomputes the FP64 residual of the GPU solution
    rel = oracle.norm(oracle.residual(u, f)) / oracle.norm(f)
    assert rel <= 1.01e-10, rel
    # final error against the oracle's FP64 solution converged from zero (to
    # 1e-13, or as far as FP64 rounding lets the residual fall at this size):
    # within the guaranteed bound (residuals of both over lambda_min(A))
    err, bound, orr = error_vs_converged_oracle(u, f, maxit=20)
    print(f"8193^2 FP32-DC: rel l2 error vs oracle {err:.3e} (bound {bound:.3e}, oracle relres {orr:.2e})")
    assert orr <= 1e-12
    assert err <= bound, (err, bound)


@pytest.mark.parametrize("n,nu1,nu2,omega", [(65, 2, 1, 1.0), (257, 1, 2, 1.2), (1025, 2, 1, 1.0), (513, 2, 2, 0.9)])
def test_fused_variable_coefficient_fp32_equals_unfused(n, nu1, nu2, omega):
    # Lognormal k (harmonic faces), FP32 inner cycles of defect correction:
    # the fused variable-stencil kernels against the one-kernel-per-operator
    # path (both round in FP32, differently), then the oracle's residual of
    # the fused path's answer after a solve to 1e-8.
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    k = synth.lognormal_k(2, n, 0x5EED0004 ^ n)
    f = synth.uniform_rhs(2, n, 0x5EED0004 ^ (n + 1))
    kw = dict(k=k, precision="fp32_dc", nu1=nu1, nu2=nu2, omega=omega)
    a, ha = history(2, n, f, 4, fuse=True, **kw)
    b, hb = history(2, n, f, 4, fuse=False, **kw)
    assert np.all(np.abs(ha - hb) <= 1e-4 * hb + 1e-12), (ha, hb)
    s = Solver(2, n, maxit=60, fuse=True, **kw)
    s.set_rhs(f)
    it, rr, _ = s.solve(1e-8)
    u = s.get_solution()
    faces = oracle.node_faces(k)
    assert oracle.norm(oracle.residual(u, f, faces=faces)) / oracle.norm(f) <= 1.01e-8


# ------------------------------------------------------------ tiling and fusion knobs

KNOBS = [dict(tile_rows=64), dict(tile_rows=8), dict(tile_max_n=1), dict(tile_max_n=2049),
         dict(fuse_depth=1), dict(fuse_depth=1, tile_max_n=1, tile_rows=128)]


@pytest.mark.parametrize("knobs", KNOBS)
@pytest.mark.parametrize("nu1,nu2,omega", [(2, 1, 1.0), (2, 2, 0.9)])
def test_tiling_knobs_fp64_match_oracle(knobs, nu1, nu2, omega):
    # Every tile shape and fusion depth computes the same FP64 iteration: the
    # per-cycle relative residuals match the oracle's to 1e-12 (1025^2 takes
    # the block tiles by default, 2049^2 the streaming kernels).
    for n in (1025, 2049):
        f = synth.uniform_rhs(2, n, 0x5EED0002 ^ n)
        _, hist = history(2, n, f, 3, nu1=nu1, nu2=nu2, omega=omega, **knobs)
        _, rho = oracle_history(2, n, f, 3, nu1=nu1, nu2=nu2, omega=omega)
        assert np.max(np.abs(hist - rho)) <= 1e-12, (knobs, n, hist, rho)


@pytest.mark.parametrize("knobs", KNOBS)
def test_tiling_knobs_fp32_dc_reach_tolerance(knobs):
    # FP32 inner cycles under every setting: the same number of outer steps to
    # 1e-10 as the default, by the oracle's own FP64 residual.
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    n = 2049
    f = synth.uniform_rhs(2, n, 0x5EED0002)
    its = []
    for kw in ({}, knobs):
        s = Solver(2, n, precision="fp32_dc", inner_cycles=3, maxit=40, **kw)
        s.set_rhs(f)
        it, rr, _ = s.solve(1e-10)
        assert oracle.norm(oracle.residual(s.get_solution(), f)) / oracle.norm(f) <= 1.01e-10
        its.append(it)
    assert its[0] == its[1]


def test_tiling_knobs_rejected_when_out_of_range():
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    from paper_1406_5369_gb300._capi import MGError
    for kw in (dict(tile_rows=-1), dict(tile_max_n=-5), dict(fuse_depth=9)):
        with pytest.raises(MGError):
            Solver(2, 65, **kw)


@pytest.mark.parametrize("n,nu1,nu2,omega,inner", [(513, 2, 1, 1.0, 3), (1025, 2, 1, 1.15, 2), (513, 1, 1, 1.0, 3),
                                                   (1025, 1, 2, 0.9, 3), (2049, 2, 1, 1.0, 4)])
def test_joined_inner_cycles_equal_separate_passes(n, nu1, nu2, omega, inner):
    # Between two inner cycles of a defect-correction step the finest inner
    # level runs post-smoothing + the next pre-smoothing as one pass
    # (join_cycles): the same FP32 operations in the same order as the two
    # separate passes, so histories and solutions agree bit for bit; the
    # oracle recomputes the final residual.
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    f = synth.uniform_rhs(2, n, 0x5EED0002 ^ n)
    out = {}
    for join in (True, False):
        s = Solver(2, n, precision="fp32_dc", nu1=nu1, nu2=nu2, omega=omega, inner_cycles=inner, maxit=30,
                   join_cycles=join)
        s.set_rhs(f)
        it, rr, hist = s.solve(1e-10)
        out[join] = (hist[: it + 1], s.get_solution(), s.kernel_launches())
    assert np.array_equal(out[True][0], out[False][0])
    assert np.array_equal(out[True][1], out[False][1])
    assert out[True][2] < out[False][2]  # fewer launches with the joined passes
    u = out[True][1]
    assert oracle.norm(oracle.residual(u, f)) / oracle.norm(f) <= 1.01e-10
