"""Batched solves of many independent problems (mg_batch_*).

Each problem of a batch must (1) match the oracle - per-step relative
residuals to 1e-12 in FP64, and the oracle's recomputed residual of the
final answer within the requested tolerance in defect correction - and
(2) give bit-for-bit the same solution alone in a batch and in a mix of
other problems of different sizes (its arithmetic, including the order of
its norm sums, does not depend on its companions).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import need_gpu, rel_err

pytestmark = pytest.mark.gpu


def make_problem(dim, m, seed, var=False, prec="fp32_dc", smoother="rbgs", omega=1.0, nu=(2, 1), inner=1, maxit=60):
    from paper_1406_5369_gb300 import Solver
    n = (1 << m) + 1
    k = synth.lognormal_k(dim, n, seed ^ 0x77) if var else None
    f = synth.uniform_rhs(dim, n, seed)
    s = Solver(dim, n, k=k, precision=prec, smoother=smoother, omega=omega, nu1=nu[0], nu2=nu[1],
               inner_cycles=inner, maxit=maxit)
    s.set_rhs(f)
    return s, f, k


def test_batched_fp64_steps_match_oracle():
    need_gpu()
    from paper_1406_5369_gb300 import BatchSolver
    ms = [5, 7, 6, 8, 5]
    probs = [make_problem(2, m, 100 + i, prec="fp64") for i, m in enumerate(ms)]
    B = BatchSolver(len(ms))
    ids = [B.add(p[0]) for p in probs]
    hist = [B.step(ids) for _ in range(5)]
    for i, (s, f, _) in enumerate(probs):
        ref = oracle.Hierarchy(2, s.n)
        ref.set_rhs(f)
        rho = ref.solve(0.0, 5)
        got = np.array([h[i] for h in hist])
        assert np.max(np.abs(got - rho[1:])) <= 1e-12, (s.n, got, rho)
        assert rel_err(s.get_solution(), ref.get_u()) <= 1e-11


def test_batched_variable_coefficient_dc_reaches_tolerance_and_mix_equals_alone():
    need_gpu()
    from paper_1406_5369_gb300 import BatchSolver
    ms = [5, 6, 7, 8, 6, 5, 7]
    probs = [make_problem(2, m, 200 + i, var=True) for i, m in enumerate(ms)]
    B = BatchSolver(len(ms))
    for p in probs:
        B.add(p[0])
    iters, rel = B.solve(1e-8, maxit=60)
    assert np.all(rel[:len(ms)] <= 1e-8)
    sols = [p[0].get_solution() for p in probs]
    for (s, f, k), u in zip(probs, sols):
        faces = oracle.node_faces(k)
        assert oracle.norm(oracle.residual(u, f, faces=faces)) / oracle.norm(f) <= 1.01e-8
    # the same problems, each alone in its own batch
    for i in (0, 3, 6):
        s, f, k = make_problem(2, ms[i], 200 + i, var=True)
        B1 = BatchSolver(1)
        B1.add(s)
        it1, rel1 = B1.solve(1e-8, maxit=60)
        assert it1[0] == iters[i]
        assert np.array_equal(s.get_solution(), sols[i])


def test_batched_3d_jacobi_dc_mix_equals_alone():
    need_gpu()
    from paper_1406_5369_gb300 import BatchSolver
    ms = [5, 4, 6, 5]
    kw = dict(smoother="jacobi", omega=6 / 7, nu=(2, 2), inner=2)
    probs = [make_problem(3, m, 300 + i, **kw) for i, m in enumerate(ms)]
    B = BatchSolver(8)
    for p in probs:
        B.add(p[0])
    tol = {0: 1e-6, 1: 1e-10, 2: 1e-10, 3: 1e-6}
    iters, rel = B.solve(tol, maxit=60)
    for i, (s, f, _) in enumerate(probs):
        assert rel[i] <= tol[i]
        u = s.get_solution()
        assert oracle.norm(oracle.residual(u, f)) / oracle.norm(f) <= 1.01 * tol[i]
    s, f, _ = make_problem(3, ms[2], 302, **kw)
    B1 = BatchSolver(1)
    B1.add(s)
    B1.solve(1e-10, maxit=60)
    assert np.array_equal(s.get_solution(), probs[2][0].get_solution())


def test_batch_argument_errors():
    need_gpu()
    from paper_1406_5369_gb300 import BatchSolver, MGError
    a, _, _ = make_problem(2, 5, 1)
    b, _, _ = make_problem(2, 5, 2, prec="fp64")
    B = BatchSolver(1)
    B.add(a)
    with pytest.raises(MGError):
        B.add(b)  # batch is full
    B2 = BatchSolver(2)
    B2.add(a)
    with pytest.raises(MGError):
        B2.add(b)  # different precision
    c, _, _ = make_problem(2, 5, 3, smoother="jacobi", omega=0.8, nu=(2, 1))
    with pytest.raises(MGError):
        BatchSolver(2).add(c)  # odd Jacobi sweeps
    with pytest.raises(MGError):
        B.step([5])
