"""The exact fixed-point outer step of defect correction.

For a constant stencil whose axis coefficients c_d / h^2 are one power of two
(Poisson with n = 2^m + 1), the FP64 outer step evaluates r = f - A u in 64-bit
fixed-point integers. The defect it writes must equal the exact residual of
the stored FP64 solution, truncated to the inner storage type, up to the
fixed-point truncation bound (1/32 of the FP64 unit in the last place of the
largest value per row, times the 2 dim + 2 dim stencil terms). The reference
residual here is computed in exact rational arithmetic from the GPU's own
FP64 solution, so the test pins the arithmetic, not just its accuracy.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from gpu_util import need_gpu, rel_err

pytestmark = pytest.mark.gpu


def exact_residual_2d(u, f, c):
    """r = f - c (4u - sum of neighbours) at interior nodes, exact rationals."""
    n = u.shape[0]
    U = [[Fraction(float(v)) for v in row] for row in u]
    r = np.zeros((n, n), dtype=object)
    C = Fraction(c)
    for j in range(1, n - 1):
        for i in range(1, n - 1):
            s = 4 * U[j][i] - U[j][i - 1] - U[j][i + 1] - U[j - 1][i] - U[j + 1][i]
            r[j, i] = Fraction(float(f[j, i])) - C * s
    return r


def one_step(n, prec, exact, u0, f, inner_cycles=1):
    from paper_1406_5369_gb300 import Solver
    s = Solver(2, n, precision=prec, maxit=1, inner_cycles=inner_cycles, exact_outer=exact)
    s.set_rhs(f)
    s.set_solution(u0)
    s.solve(0.0, raise_on_noconv=False)
    return s, s.get_solution(), s.get_field(0, "f"), s.get_field(0, "u")


@pytest.mark.parametrize("prec", ["fp32_dc", "bf16_dc"])
@pytest.mark.parametrize("n", [33, 65])
def test_exact_defect_is_truncated_exact_residual(prec, n):
    need_gpu()
    rng = np.random.default_rng(n)
    f = synth.uniform_rhs(2, n, 0x5EED0002 ^ n)
    # an initial guess with structure over several binades and sign changes
    x = np.linspace(0.0, 1.0, n)
    u0 = np.outer(np.sin(3 * np.pi * x), np.sin(2 * np.pi * x)) * 1e-3
    u0[1:-1, 1:-1] += 1e-7 * rng.standard_normal((n - 2, n - 2))
    u0[0, :] = u0[-1, :] = u0[:, 0] = u0[:, -1] = 0.0
    s, u, d, e = one_step(n, prec, True, u0, f)
    # the update is one IEEE FP64 addition per node
    assert np.array_equal(u[1:-1, 1:-1], u0[1:-1, 1:-1] + e[1:-1, 1:-1])
    c = float((n - 1) ** 2)
    r = exact_residual_2d(u, f, c)
    ri = np.array([[float(r[j, i]) for i in range(1, n - 1)] for j in range(1, n - 1)])
    di = d[1:-1, 1:-1]
    # truncation to the inner type: 2^-23 relative (FP32), 2^-8 (BF16 rounds the truncated FP32)
    rel = 2.0 ** -23 if prec == "fp32_dc" else 2.0 ** -8 + 2.0 ** -22
    abs_fix = 12 * c * np.max(np.abs(u)) * 2.0 ** -56 + np.max(np.abs(f)) * 2.0 ** -56
    err = np.abs(di - ri)
    bound = rel * np.abs(ri) * 1.0000001 + abs_fix
    assert np.all(err <= bound), float(np.max(err - bound))
    # the FP64-arithmetic kernel makes the same update; its defect differs by
    # the truncation to the inner type and its own FP64 rounding at most
    _, u64, d64, _ = one_step(n, prec, False, u0, f)
    assert np.array_equal(u64, u)
    fp64_noise = 16 * c * np.max(np.abs(u)) * 2.0 ** -52
    assert np.all(np.abs(d64[1:-1, 1:-1] - di) <= 2 * rel * np.abs(ri) * 1.0000001 + fp64_noise + abs_fix)


@pytest.mark.parametrize("n", [1025, 2049])
def test_exact_outer_solve_matches_fp64_outer(n):
    # Whole FP32-DC solves to 1e-10 with the exact and the FP64-arithmetic
    # outer step: same number of outer steps, both reach the tolerance by the
    # oracle's own FP64 residual, solutions agree to the solve tolerance.
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    f = synth.uniform_rhs(2, n, 0x5EED0002)
    res = {}
    for exact in (True, False):
        s = Solver(2, n, precision="fp32_dc", inner_cycles=3, maxit=40, exact_outer=exact)
        s.set_rhs(f)
        it, rr, hist = s.solve(1e-10)
        u = s.get_solution()
        rel = oracle.norm(oracle.residual(u, f)) / oracle.norm(f)
        assert rel <= 1.01e-10, (exact, rel)
        res[exact] = (it, hist[: it + 1], u)
    assert res[True][0] == res[False][0]
    # the first outer step's norm sees the same solution up to FP32 rounding of the defect
    assert abs(res[True][1][1] - res[False][1][1]) <= 1e-5 * res[False][1][1]
    assert rel_err(res[True][2], res[False][2]) <= 1e-8


def test_exact_outer_only_for_power_of_two_stencils():
    # An anisotropic stencil (cx != cy) keeps the FP64-arithmetic outer step;
    # both settings then give bit-identical solves.
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    n = 257
    f = synth.uniform_rhs(2, n, 11)
    out = []
    for exact in (True, False):
        s = Solver(2, n, stencil=(1.0, 0.5, 1.0), precision="fp32_dc", maxit=30, exact_outer=exact)
        s.set_rhs(f)
        it, rr, hist = s.solve(1e-10)
        out.append((hist[: it + 1], s.get_solution()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_exact_outer_with_dirichlet_data():
    # Non-zero boundary values take part in the row exponents and the stencil.
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    n = 513
    x = np.linspace(0.0, 1.0, n)
    g = 1.0 + np.add.outer(x, 2 * x)
    g[1:-1, 1:-1] = 0.0
    f = synth.uniform_rhs(2, n, 23)
    s = Solver(2, n, dirichlet=g, precision="fp32_dc", maxit=40)
    s.set_rhs(f)
    it, rr, _ = s.solve(1e-10)
    u = s.get_solution()
    r0 = oracle.residual(g, f)
    rel = oracle.norm(oracle.residual(u, f)) / oracle.norm(r0)
    assert rel <= 1.01e-10, rel


def exact_residual_3d(u, f, c):
    """r = f - c (6u - sum of the six neighbours) at interior nodes, exact rationals."""
    n = u.shape[0]
    U = np.vectorize(lambda v: Fraction(float(v)), otypes=[object])(u)
    C = Fraction(c)
    r = np.zeros((n, n, n))
    for k in range(1, n - 1):
        for j in range(1, n - 1):
            for i in range(1, n - 1):
                s = (6 * U[k, j, i] - U[k, j, i - 1] - U[k, j, i + 1] - U[k, j - 1, i] - U[k, j + 1, i]
                     - U[k - 1, j, i] - U[k + 1, j, i])
                r[k, j, i] = float(Fraction(float(f[k, j, i])) - C * s)
    return r


@pytest.mark.parametrize("prec", ["fp32_dc", "bf16_dc"])
def test_exact_defect_3d_is_truncated_exact_residual(prec):
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    n = 17
    rng = np.random.default_rng(5)
    f = synth.normal_rhs(3, n, 0x5EED0003)
    x = np.linspace(0.0, 1.0, n)
    u0 = np.einsum("i,j,k->kji", np.sin(np.pi * x), np.sin(2 * np.pi * x), np.sin(3 * np.pi * x)) * 1e-2
    u0[1:-1, 1:-1, 1:-1] += 1e-6 * rng.standard_normal((n - 2,) * 3)
    u0[0], u0[-1], u0[:, 0], u0[:, -1], u0[:, :, 0], u0[:, :, -1] = 0, 0, 0, 0, 0, 0
    out = {}
    for exact in (True, False):
        s = Solver(3, n, precision=prec, smoother="jacobi", omega=6 / 7, nu1=2, nu2=2, maxit=1, exact_outer=exact)
        s.set_rhs(f)
        s.set_solution(u0)
        s.solve(0.0, raise_on_noconv=False)
        out[exact] = (s.get_solution(), s.get_field(0, "f"), s.get_field(0, "u"))
    u, d, e = out[True]
    inner = (slice(1, -1),) * 3
    assert np.array_equal(u[inner], u0[inner] + e[inner])
    assert np.array_equal(out[False][0], u)
    c = float((n - 1) ** 2)
    r = exact_residual_3d(u, f, c)
    rel = 2.0 ** -23 if prec == "fp32_dc" else 2.0 ** -8 + 2.0 ** -22
    abs_fix = 16 * c * np.max(np.abs(u)) * 2.0 ** -56 + np.max(np.abs(f)) * 2.0 ** -56
    err = np.abs(d[inner] - r[inner])
    assert np.all(err <= rel * np.abs(r[inner]) * 1.0000001 + abs_fix), float(np.max(err))
    fp64_noise = 24 * c * np.max(np.abs(u)) * 2.0 ** -52
    assert np.all(np.abs(out[False][1][inner] - d[inner]) <= 2 * rel * np.abs(r[inner]) * 1.0000001 + fp64_noise + abs_fix)


@pytest.mark.parametrize("prec", ["fp32_dc", "bf16_dc"])
def test_exact_outer_3d_solve_matches_fp64_outer(prec):
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    n = 129
    f = synth.normal_rhs(3, n, 0x5EED0003)
    res = {}
    for exact in (True, False):
        s = Solver(3, n, precision=prec, smoother="jacobi", omega=6 / 7, nu1=2, nu2=2, inner_cycles=3, maxit=40,
                   exact_outer=exact)
        s.set_rhs(f)
        it, rr, hist = s.solve(1e-10)
        u = s.get_solution()
        rel = oracle.norm(oracle.residual(u, f)) / oracle.norm(f)
        assert rel <= 1.01e-10, (exact, rel)
        res[exact] = (it, u)
    assert res[True][0] == res[False][0]
    assert rel_err(res[True][1], res[False][1]) <= 1e-8


@pytest.mark.parametrize("prec", ["fp32_dc", "bf16_dc"])
def test_exact_defect_3d_multi_tile_matches_fp64_outer(prec):
    # 257^3: two 128-column x-tiles, 32 y-tiles with a ragged last one, several
    # z-chunks. One outer step from a structured u0: the exact kernel's update
    # is the FP64 kernel's bit for bit, and the two defects differ by at most
    # the inner-type truncation of each, the FP64 kernel's own rounding and
    # the fixed-point truncation bound (global max |u| scale).
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    n = 257
    rng = np.random.default_rng(7)
    f = synth.normal_rhs(3, n, 0x5EED0103)
    x = np.linspace(0.0, 1.0, n)
    u0 = np.einsum("i,j,k->kji", np.sin(np.pi * x), np.sin(2 * np.pi * x), np.sin(3 * np.pi * x)) * 1e-2
    u0[1:-1, 1:-1, 1:-1] += 1e-6 * rng.standard_normal((n - 2,) * 3)
    u0[0], u0[-1], u0[:, 0], u0[:, -1], u0[:, :, 0], u0[:, :, -1] = 0, 0, 0, 0, 0, 0
    out = {}
    for exact in (True, False):
        s = Solver(3, n, precision=prec, smoother="jacobi", omega=6 / 7, nu1=2, nu2=2, maxit=1, exact_outer=exact)
        s.set_rhs(f)
        s.set_solution(u0)
        s.solve(0.0, raise_on_noconv=False)
        out[exact] = (s.get_solution(), s.get_field(0, "f"))
        del s
    inner = (slice(1, -1),) * 3
    u, d = out[True]
    u64, d64 = out[False]
    assert np.array_equal(u, u64)
    c = float((n - 1) ** 2)
    rel = 2.0 ** -23 if prec == "fp32_dc" else 2.0 ** -8 + 2.0 ** -22
    abs_fix = 16 * c * np.max(np.abs(u)) * 2.0 ** -56 + np.max(np.abs(f)) * 2.0 ** -56
    fp64_noise = 24 * c * np.max(np.abs(u)) * 2.0 ** -52
    ref = np.abs(d64[inner])
    err = np.abs(d[inner] - d64[inner])
    assert np.all(err <= 2.01 * rel * ref + fp64_noise + abs_fix), float(np.max(err - 2.01 * rel * ref))
    assert np.all(d[0] == 0) and np.all(d[:, :, -1] == 0)
