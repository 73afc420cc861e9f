"""Dense coarsest-grid solve (coarsest_n = 5 or 9) against the FP64 oracle.

With coarsest_n > 3 the coarsest grid keeps (coarsest_n - 2)^dim unknowns
and is solved directly (Algorithm 1, coarsest level): the library forms the
FP64 inverse of the coarsest operator once at creation (Gauss-Jordan
elimination in one block) and applies it to the residual; the oracle factors
the same matrix by Gaussian elimination with partial pivoting. Both are exact
solves of one system with condition number below 40, so from a zero start
they agree to roughly 1e-15 (the tests allow 1e-13; a nonzero start adds the
rounding of its residual, bounded in the test). V-cycle histories agree with the
oracle's to 1e-12 per cycle, as for the 3^dim coarsest grid, on both routes
to the coarsest grid (the per-operator kernels, fuse=False, and the
single-block coarse cycle, fuse=True), and a problem gives the same result in
a batch as alone.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import need_gpu, rel_err, zero_boundary

pytestmark = pytest.mark.gpu

CASES = [(2, 5), (2, 9), (3, 5), (3, 9)]
FINE = {2: 65, 3: 17}


def solver(dim, n, nc, **kw):
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    return Solver(dim, n, coarsest_n=nc, **kw)


@pytest.mark.parametrize("dim,nc", CASES)
@pytest.mark.parametrize("var", [False, True])
def test_coarse_solve_is_the_dense_solution(dim, nc, var):
    n = FINE[dim]
    k = synth.lognormal_k(dim, n, 0x5EED0004) if var else None
    s = solver(dim, n, nc, k=k)
    ref = oracle.Hierarchy(dim, n, knode=k, coarsest_n=nc)
    l = s.levels - 1
    assert s.level_size(l) == nc and ref.level_n(l) == nc
    s.set_field(l, "f", zero_boundary(synth.uniform(13, (nc,) * dim)))
    f = s.get_field(l, "f")
    want = oracle.dense_solve(f, faces=ref.faces(l))
    s.set_field(l, "u", np.zeros((nc,) * dim))
    s.coarse_solve()
    assert rel_err(s.get_field(l, "u"), want) <= 1e-13
    # From a nonzero start u0 the step u0 + A^{-1}(f - A u0) carries the
    # rounding of f - A u0 through A^{-1}: relative error up to about
    # eps * cond(A) * (max|u0| / max|u| + 1), cond(A) < 40 on these grids.
    u0 = zero_boundary(synth.uniform(17, (nc,) * dim))
    s.set_field(l, "u", u0)
    s.coarse_solve()
    bound = 32 * np.finfo(float).eps * 40 * (np.max(np.abs(u0)) / np.max(np.abs(want)) + 1)
    assert rel_err(s.get_field(l, "u"), want) <= bound


@pytest.mark.parametrize("dim,nc", CASES)
@pytest.mark.parametrize("var", [False, True])
@pytest.mark.parametrize("fuse", [True, False])
def test_vcycle_history_matches_oracle(dim, nc, var, fuse):
    n = {2: 129, 3: 33}[dim]
    k = synth.lognormal_k(dim, n, 0x5EED0004 ^ nc) if var else None
    f = synth.uniform_rhs(dim, n, 0x5EED0002 + nc)
    if dim == 2:
        sm = dict(smoother="rbgs", omega=1.0, nu1=2, nu2=1)
    else:
        sm = dict(smoother="jacobi", omega=6 / 7, nu1=2, nu2=2)
    s = solver(dim, n, nc, k=k, maxit=6, fuse=fuse, **sm)
    s.set_rhs(f)
    _, _, hist = s.solve(0.0, raise_on_noconv=False)
    ref = oracle.Hierarchy(dim, n, knode=k, coarsest_n=nc, smoother=0 if sm["smoother"] == "rbgs" else 1,
                           omega=sm["omega"], nu1=sm["nu1"], nu2=sm["nu2"])
    ref.set_rhs(f)
    rho = ref.solve(0.0, 6)
    assert len(hist) == len(rho)
    assert np.max(np.abs(hist - rho)) <= 1e-12, (hist, rho)
    assert rel_err(s.get_solution(), ref.get_u()) <= 1e-11


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("fuse", [True, False])
def test_single_level_problem_is_solved_in_one_cycle(dim, fuse):
    # n == coarsest_n: the hierarchy is the coarsest grid alone, with
    # Dirichlet values on its boundary
    n = 9
    f = synth.uniform_rhs(dim, n, 0x5EED0009)
    g = synth.uniform(19, (n,) * dim)
    s = solver(dim, n, n, dirichlet=g, maxit=1, fuse=fuse)
    assert s.levels == 1
    s.set_rhs(f)
    _, rr, _ = s.solve(0.0, raise_on_noconv=False)
    assert rr <= 1e-14
    ub = g.copy()
    ub[(slice(1, -1),) * dim] = 0.0
    want = oracle.dense_solve(f, u_boundary=ub)
    assert rel_err(s.get_solution(), want) <= 1e-13


@pytest.mark.parametrize("prec", ["fp32_dc", "bf16_dc"])
def test_defect_correction_with_dense_coarsest_reaches_tolerance(prec):
    n = 257
    k = synth.lognormal_k(2, n, 0x5EED0004)
    f = synth.uniform_rhs(2, n, 0x5EED0004)
    s = solver(2, n, 9, k=k, precision=prec, maxit=40)
    s.set_rhs(f)
    _, rr, _ = s.solve(1e-10)
    assert rr <= 1e-10
    ref = oracle.Hierarchy(2, n, knode=k, coarsest_n=9)
    ref.set_rhs(f)
    r0 = ref.residual_norm()
    ref.set_u(s.get_solution())
    assert ref.residual_norm() <= 1.05e-10 * r0


def test_batch_mixes_coarsest_sizes_and_equals_alone():
    need_gpu()
    from paper_1406_5369_gb300 import BatchSolver
    specs = [(6, 5), (7, 3), (5, 9), (8, 5), (6, 9)]

    def make(m, nc, seed):
        n = (1 << m) + 1
        s = solver(2, n, nc, k=synth.lognormal_k(2, n, seed), precision="fp32_dc", maxit=40)
        s.set_rhs(synth.uniform_rhs(2, n, seed))
        return s

    mixed = [make(m, nc, 300 + i) for i, (m, nc) in enumerate(specs)]
    B = BatchSolver(len(specs))
    for s in mixed:
        B.add(s)
    _, rel = B.solve(1e-9)
    assert np.all(rel[:len(specs)] <= 1e-9)
    for i, (m, nc) in enumerate(specs):
        alone = make(m, nc, 300 + i)
        A = BatchSolver(1)
        A.add(alone)
        A.solve(1e-9)
        assert np.array_equal(alone.get_solution(), mixed[i].get_solution())
