"""Whole-solver parity of the CUDA library with the FP64 oracle.

FP64: the relative residual rho_k = ||r_k|| / ||r_0|| of every V-cycle agrees
with the oracle's to 1e-12 (absolute), and the final solutions agree to
1e-11 relative. Reduced-precision defect correction (FP32 / BF16 inner
cycles, FP64 outer loop) must reach the requested tolerance; its final
solution is compared with the oracle's converged FP64 solution, and the
oracle recomputes the residual of the GPU's solution itself.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import need_gpu, rel_err

pytestmark = pytest.mark.gpu

RHO_TOL = 1e-12


def run_pair(dim, n, f, *, smoother="rbgs", omega=1.0, nu1=2, nu2=1, k=None, dirichlet=None,
             stencil=(1.0, 1.0, 1.0), cycles=10, use_graph=True, u0=None):
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    s = Solver(dim, n, k=k, dirichlet=dirichlet, stencil=stencil, smoother=smoother, omega=omega,
               nu1=nu1, nu2=nu2, maxit=cycles, use_graph=use_graph)
    s.set_rhs(f)
    if u0 is not None:
        s.set_solution(u0)
    it, rr, hist = s.solve(0.0, raise_on_noconv=False)
    ref = oracle.Hierarchy(dim, n, c=stencil, knode=k, smoother=0 if smoother == "rbgs" else 1,
                           omega=omega, nu1=nu1, nu2=nu2)
    ref.set_rhs(f)
    ub = np.zeros((n,) * dim) if dirichlet is None else dirichlet.copy()
    if dirichlet is not None:
        ub[(slice(1, -1),) * dim] = 0.0
    if u0 is not None:
        ub[(slice(1, -1),) * dim] = u0[(slice(1, -1),) * dim]
    ref.set_u(ub)
    rho = ref.solve(0.0, cycles)
    return s, ref, hist, rho


def check_history(hist, rho):
    assert len(hist) == len(rho), (len(hist), len(rho))
    d = np.max(np.abs(hist - rho))
    assert d <= RHO_TOL, (d, hist, rho)


@pytest.mark.parametrize("use_graph", [True, False])
def test_config1_poisson_129(use_graph):
    # 2D Poisson, 129^2, f = 2 pi^2 sin sin, V(2,1) RBGS omega 1, 10 cycles from 0.
    n = 129
    f = synth.sine_rhs(2, n)
    s, ref, hist, rho = run_pair(2, n, f, cycles=10, use_graph=use_graph)
    assert s.levels == 7
    check_history(hist, rho)
    u = s.get_solution()
    assert rel_err(u, ref.get_u()) <= 1e-11
    h = 1.0 / (n - 1)
    ch = (math.pi * h / 2) ** 2 / math.sin(math.pi * h / 2) ** 2
    assert abs(np.max(np.abs(u - synth.sine_solution(2, n))) - (ch - 1)) < 1e-7


@pytest.mark.parametrize("n", [3, 5, 9, 17, 33, 513])
def test_poisson_2d_sizes(n):
    f = synth.uniform_rhs(2, n, 0x5EED0002)
    _, _, hist, rho = run_pair(2, n, f, cycles=8)
    check_history(hist, rho)


@pytest.mark.parametrize("n,smoother,omega,nu", [(33, "jacobi", 6 / 7, (2, 2)), (65, "jacobi", 6 / 7, (2, 2)),
                                                 (33, "rbgs", 1.0, (2, 1)), (5, "jacobi", 0.8, (1, 1))])
def test_poisson_3d(n, smoother, omega, nu):
    f = synth.normal_rhs(3, n, 0x5EED0003)
    _, _, hist, rho = run_pair(3, n, f, smoother=smoother, omega=omega, nu1=nu[0], nu2=nu[1], cycles=8)
    check_history(hist, rho)


@pytest.mark.parametrize("dim,n,smoother", [(2, 129, "rbgs"), (2, 65, "jacobi"), (3, 33, "jacobi"), (3, 17, "rbgs")])
def test_variable_coefficient(dim, n, smoother):
    k = synth.lognormal_k(dim, n, 0x5EED0004)
    f = synth.uniform_rhs(dim, n, 0x5EED0004 ^ 1)
    omega = 1.0 if smoother == "rbgs" else 0.8
    s, ref, hist, rho = run_pair(dim, n, f, k=k, smoother=smoother, omega=omega, cycles=8)
    check_history(hist, rho)
    assert rel_err(s.get_solution(), ref.get_u()) <= 1e-11


def test_dirichlet_values_and_initial_guess():
    n = 65
    g = synth.uniform(21, (n, n))
    f = synth.uniform_rhs(2, n, 22)
    u0 = synth.random_u0(2, n, 23)
    s, ref, hist, rho = run_pair(2, n, f, dirichlet=g, u0=u0, cycles=6)
    check_history(hist, rho)
    u = s.get_solution()
    assert np.array_equal(u[0], g[0]) and np.array_equal(u[:, -1], g[:, -1])
    assert rel_err(u, ref.get_u()) <= 1e-11


def test_anisotropic_constant_stencil():
    n = 65
    f = synth.uniform_rhs(2, n, 24)
    _, _, hist, rho = run_pair(2, n, f, stencil=(1.0, 0.25, 1.0), cycles=6)
    check_history(hist, rho)


def test_jacobi_odd_sweeps_with_graph_replay():
    # nu1 + nu2 odd flips the live buffer each cycle, so the replayed graphs
    # alternate between two captures.
    n = 65
    f = synth.uniform_rhs(2, n, 25)
    _, _, hist, rho = run_pair(2, n, f, smoother="jacobi", omega=0.8, nu1=2, nu2=1, cycles=7)
    check_history(hist, rho)


def test_single_level_grid_is_exact():
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    for dim in (2, 3):
        s = Solver(dim, 3, maxit=2)
        f = np.zeros((3,) * dim)
        f[(1,) * dim] = 5.0
        s.set_rhs(f)
        it, rr, _ = s.solve(1e-14)
        assert it == 1 and rr <= 1e-14


def test_vcycle_call_matches_solve_step():
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    n = 129
    f = synth.uniform_rhs(2, n, 26)
    a = Solver(2, n, maxit=3)
    a.set_rhs(f)
    a.solve(0.0, raise_on_noconv=False)
    b = Solver(2, n)
    b.set_rhs(f)
    for _ in range(3):
        b.vcycle()
    assert np.array_equal(a.get_solution(), b.get_solution())


# ---------------------------------------------------------------- defect correction

def oracle_solution(dim, n, f, k=None, smoother=0, omega=1.0, nu=(2, 1)):
    ref = oracle.Hierarchy(dim, n, knode=k, smoother=smoother, omega=omega, nu1=nu[0], nu2=nu[1])
    ref.set_rhs(f)
    ref.solve(1e-13, 60)
    return ref


@pytest.mark.parametrize("prec,dim,n,smoother,omega,nu,tol,err_bound", [
    ("fp32_dc", 2, 513, "rbgs", 1.0, (2, 1), 1e-10, 1e-9),
    ("bf16_dc", 2, 257, "rbgs", 1.0, (2, 1), 1e-10, 1e-9),
    ("fp32_dc", 3, 65, "jacobi", 6 / 7, (2, 2), 1e-10, 1e-9),
    ("bf16_dc", 3, 65, "jacobi", 6 / 7, (2, 2), 1e-10, 1e-9),
])
def test_defect_correction_reaches_tolerance(prec, dim, n, smoother, omega, nu, tol, err_bound):
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    f = synth.uniform_rhs(dim, n, 0x5EED0002) if dim == 2 else synth.normal_rhs(dim, n, 0x5EED0003)
    s = Solver(dim, n, precision=prec, smoother=smoother, omega=omega, nu1=nu[0], nu2=nu[1], maxit=60)
    s.set_rhs(f)
    it, rr, hist = s.solve(tol)
    assert rr <= tol
    u = s.get_solution()
    # the oracle recomputes the relative residual of the GPU's answer itself
    r_rel = oracle.norm(oracle.residual(u, f)) / oracle.norm(oracle.residual(np.zeros_like(f), f))
    assert r_rel <= 1.01 * tol, r_rel
    ref = oracle_solution(dim, n, f, smoother=0 if smoother == "rbgs" else 1, omega=omega, nu=nu)
    assert rel_err(u, ref.get_u()) <= err_bound


def test_defect_correction_variable_coefficient():
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    n = 257
    k = synth.lognormal_k(2, n, 0x5EED0004)
    f = synth.uniform_rhs(2, n, 0x5EED0005)
    s = Solver(2, n, k=k, precision="fp32_dc", maxit=60)
    s.set_rhs(f)
    it, rr, _ = s.solve(1e-8)
    u = s.get_solution()
    faces = oracle.node_faces(k)
    r_rel = oracle.norm(oracle.residual(u, f, faces=faces)) / oracle.norm(f)
    assert r_rel <= 1.01e-8
    ref = oracle_solution(2, n, f, k=k)
    assert rel_err(u, ref.get_u()) <= 1e-6


def test_fp64_cycle_of_defect_correction_shape_matches_plain():
    # The oracle's FP64 defect correction reproduces the plain iteration; the
    # FP32 inner form stays within FP32 rounding of the same history early on.
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    n = 257
    f = synth.uniform_rhs(2, n, 31)
    s = Solver(2, n, precision="fp32_dc", maxit=4)
    s.set_rhs(f)
    _, _, hist = s.solve(0.0, raise_on_noconv=False)
    ref = oracle.Hierarchy(2, n)
    ref.set_rhs(f)
    rho = ref.dc_solve(0.0, 4)
    assert len(hist) == len(rho)
    assert np.all(np.abs(hist - rho) <= 1e-5 * rho + 1e-12)


@pytest.mark.parametrize("prec", ["fp32_dc", "bf16_dc"])
def test_defect_correction_several_inner_cycles(prec):
    # inner_cycles = 2: e = V(V(0, d), d) per outer FP64 step; fewer outer
    # steps to the same FP64 residual, which the oracle recomputes.
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    n = 1025
    f = synth.uniform_rhs(2, n, 0x5EED0002)
    its = {}
    for ic in (1, 2):
        s = Solver(2, n, precision=prec, inner_cycles=ic, maxit=60)
        s.set_rhs(f)
        it, rr, _ = s.solve(1e-10)
        assert rr <= 1e-10
        u = s.get_solution()
        assert oracle.norm(oracle.residual(u, f)) / oracle.norm(f) <= 1.01e-10
        its[ic] = it
    assert its[2] < its[1]


def test_kernel_timing_instrumentation():
    # Events bracket every launch, inside replayed graphs too; totals are
    # positive for the classes a DC solve runs and counts follow the launches.
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    n = 1025
    f = synth.uniform_rhs(2, n, 7)
    s = Solver(2, n, precision="fp32_dc", inner_cycles=2, maxit=30)
    s.set_rhs(f)
    s.set_timing(True)
    it, rr, _ = s.solve(1e-10)
    pre_ms, pre_n = s.timing("pre", 0)
    post_ms, post_n = s.timing("post", 0)
    pp_ms, pp_n = s.timing("postpre", 0)
    out_ms, out_n = s.timing("outer", 0)
    # with 2 inner cycles per step, level 0 runs a pre-smoothing pass, one
    # joined post + pre pass and a post-smoothing pass per step
    assert pre_n == post_n == pp_n == it and pre_ms > 0 and post_ms > 0 and pp_ms > 0
    # one outer step per iteration (the first residual of a zero start is f,
    # formed by a norm pass)
    assert out_n == it and out_ms > 0
    assert s.timing("pre", 1)[1] == 2 * it
    s.reset_timing()
    assert s.timing("pre", 0) == (0.0, 0)
    # level-0-only mode: the finest level and the outer step, nothing below
    s.set_timing(True, level0_only=True)
    s.set_solution(None)
    it2, _, _ = s.solve(1e-10)
    assert s.timing("pre", 0)[1] == it2 and s.timing("postpre", 0)[1] == it2 and s.timing("outer", 0)[1] == it2
    assert s.timing("pre", 1) == (0.0, 0) and s.timing("coarse", s.levels - 1) == (0.0, 0)
    # outer-only mode: the outer step alone
    s.set_timing(True, outer_only=True)
    s.reset_timing()
    s.set_solution(None)
    it3, _, _ = s.solve(1e-10)
    assert s.timing("outer", 0)[1] == it3 and s.timing("outer", 0)[0] > 0
    assert s.timing("pre", 0) == (0.0, 0) and s.timing("postpre", 0) == (0.0, 0) and s.timing("post", 0) == (0.0, 0)
    s.set_timing(False)
    s.reset_timing()
    s.set_solution(None)
    s.solve(1e-10)
    assert s.timing("pre", 0) == (0.0, 0)
