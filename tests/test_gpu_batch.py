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


def _solve_batch(probs, tol, maxit, capture, inner=None):
    from paper_1406_5369_gb300 import BatchSolver
    B = BatchSolver(len(probs) + 1)
    for p in probs:
        p[0].set_solution(None)
        B.add(p[0])
    if inner:
        B.set_inner_cycles(inner)
    B.set_capture(capture)
    iters, rel = B.solve(tol, maxit=maxit, raise_on_noconv=False)
    sols = [p[0].get_solution() for p in probs]
    launches = B.launches()
    B.close()
    return iters, rel, sols, launches


@pytest.mark.parametrize("case", ["2d_var_fp32", "2d_fp64", "3d_jacobi_bf16", "3d_rbgs_fp32"])
def test_captured_solve_equals_stepped_solve(case):
    """mg_batch_solve replaying two captured steps (stopping test on the
    device, converged problems skipped by every later launch) gives the same
    steps, ratios and solutions, bit for bit, as one mg_batch_step per step.
    Tolerances are mixed so that problems stop after odd and even step counts
    while others go on (the buffer state after an odd count is the one of the
    first captured step)."""
    need_gpu()
    if case == "2d_var_fp32":
        ms, mk = [5, 7, 6, 8, 5, 9], dict(var=True)
    elif case == "2d_fp64":
        ms, mk = [5, 6, 7, 6], dict(prec="fp64")
    elif case == "3d_jacobi_bf16":
        ms, mk = [4, 5, 6, 5], dict(prec="bf16_dc", smoother="jacobi", omega=6 / 7, nu=(2, 2), inner=2)
    else:
        ms, mk = [4, 5, 5], dict(prec="fp32_dc")
    dim = 3 if case.startswith("3d") else 2
    tols = [1e-6, 1e-10, 1e-8, 1e-4, 1e-10, 1e-7]
    tol = {i: tols[i % len(tols)] for i in range(len(ms))}
    out = {}
    for capture in (False, True):
        probs = [make_problem(dim, m, 500 + i, **mk) for i, m in enumerate(ms)]
        out[capture] = _solve_batch(probs, tol, 60, capture)
    (i0, r0, s0, l0), (i1, r1, s1, l1) = out[False], out[True]
    n = len(ms)
    assert np.array_equal(i0[:n], i1[:n]), (i0[:n], i1[:n])
    assert np.array_equal(r0[:n], r1[:n])
    if case == "2d_var_fp32":  # odd and even step counts both occur in this mix
        assert len(set(int(x) % 2 for x in i1[:n])) == 2, i1[:n]
    for a, b in zip(s0, s1):
        assert np.array_equal(a, b)
    assert all(r1[i] <= tol[i] for i in range(n))
    assert l1 > 0


def test_captured_solve_stops_at_maxit_and_reports_noconv():
    need_gpu()
    from paper_1406_5369_gb300 import MGError
    probs = [make_problem(2, m, 600 + i, var=True) for i, m in enumerate([6, 7, 5])]
    for maxit in (3, 4):
        outs = []
        for capture in (False, True):
            for p in probs:
                p[0].set_solution(None)
            outs.append(_solve_batch(probs, 1e-14, maxit, capture))
        (i0, r0, s0, _), (i1, r1, s1, _) = outs
        assert np.all(i1[:3] == maxit) and np.array_equal(i0[:3], i1[:3]) and np.array_equal(r0[:3], r1[:3])
        for a, b in zip(s0, s1):
            assert np.array_equal(a, b)
    from paper_1406_5369_gb300 import BatchSolver
    B = BatchSolver(2)
    for p in probs[:2]:
        p[0].set_solution(None)
        B.add(p[0])
    with pytest.raises(MGError):
        B.solve(1e-14, maxit=2)


def test_batch_kernel_timing_counts_groups_and_bytes_without_changing_results():
    """mg_batch_set_timing brackets each launch group with CUDA events: the
    solve with timing on gives the same bits as with it off, every kind that
    ran reports launch groups, positive time and the operator-model bytes
    (for one 2D FP32 constant-stencil problem: the level-0 pre-smoothing pass
    from zero moves 2.25 words per node)."""
    need_gpu()
    outs = []
    for timing in (False, True):
        from paper_1406_5369_gb300 import BatchSolver
        s, f, _ = make_problem(2, 9, 700)
        B = BatchSolver(2)
        B.add(s)
        B.set_capture(False)
        B.set_timing(timing)
        it, rel = B.solve(1e-8, maxit=30)
        outs.append((it[0], s.get_solution()))
        if timing:
            for kind in ("pre", "post", "coarse", "outer"):
                ms, n, by = B.timing(kind)
                assert n > 0 and ms > 0, kind
            ms, n, by = B.timing("pre")
            n0 = 513 * 513
            # levels 513, 257, 129 run the fused kernels from zero in each inner cycle (inner = 1 here)
            per_cycle = 2.25 * 4 * (513 ** 2 + 257 ** 2 + 129 ** 2)
            assert by == pytest.approx(per_cycle * it[0], rel=1e-12), (by, per_cycle * it[0])
            B.reset_timing()
            assert B.timing("pre") == (0.0, 0, 0.0)
    assert outs[0][0] == outs[1][0] and np.array_equal(outs[0][1], outs[1][1])


def test_async_steps_on_two_streams_equal_synchronous_steps():
    """mg_batch_step_async / mg_batch_step_wait on a 2D and a 3D batch, each
    on a stream of its own and both in flight at once, give the same ratios
    and solutions, bit for bit, as mg_batch_step; a problem added while a step
    is in flight joins the next step; misuse is refused."""
    torch = need_gpu()
    from paper_1406_5369_gb300 import BatchSolver, MGError
    kw3 = dict(prec="bf16_dc", smoother="jacobi", omega=6 / 7, nu=(2, 2), inner=2)

    def make_all():
        p2 = [make_problem(2, m, 800 + i, inner=3) for i, m in enumerate([6, 8, 7])]
        p3 = [make_problem(3, m, 850 + i, **kw3) for i, m in enumerate([5, 4])]
        return p2, p3

    # synchronous reference
    p2, p3 = make_all()
    B2, B3 = BatchSolver(4), BatchSolver(4)
    i2 = [B2.add(p[0]) for p in p2]
    i3 = [B3.add(p[0]) for p in p3]
    ref = [(B2.step(i2), B3.step(i3)) for _ in range(4)]
    ref_u = [p[0].get_solution() for p in p2 + p3]
    # asynchronous, two streams
    q2, q3 = make_all()
    s2, s3 = torch.cuda.Stream(), torch.cuda.Stream()
    A2, A3 = BatchSolver(4, stream=s2.cuda_stream), BatchSolver(4, stream=s3.cuda_stream)
    j2 = [A2.add(p[0]) for p in q2]
    j3 = [A3.add(p[0]) for p in q3]
    for k in range(4):
        A2.step_async(j2)
        A3.step_async(j3)
        with pytest.raises(MGError):
            A2.step_async(j2)  # one step in flight per batch
        r3 = A3.step_wait()
        r2 = A2.step_wait()
        assert np.array_equal(r2, ref[k][0]) and np.array_equal(r3, ref[k][1]), k
    with pytest.raises(MGError):
        A2.step_wait()  # nothing in flight
    for p, u in zip(q2 + q3, ref_u):
        assert np.array_equal(p[0].get_solution(), u)
    # a problem added while a step runs takes its first step with the next one
    late, f_late, _ = make_problem(2, 6, 800, inner=3)
    A2.step_async(j2)
    jl = A2.add(late)
    A2.step_wait()
    A2.step_async([jl])
    rl = A2.step_wait()
    fresh, _, _ = make_problem(2, 6, 800, inner=3)
    B1 = BatchSolver(1)
    B1.add(fresh)
    assert np.array_equal(rl, B1.step([0]))


def test_zero_start_first_defect_in_batches():
    """A problem that starts from u = 0 under homogeneous Dirichlet data gets
    the residual f itself as its first defect (no stencil pass), a problem
    with a non-zero start the full residual; both first norms are the
    oracle's (the first step's ratio uses them). After a batch step the
    solution is no longer zero, so a single-context solve that follows forms
    the full residual of it."""
    need_gpu()
    from paper_1406_5369_gb300 import BatchSolver
    for dim, m, prec in ((2, 7, "fp32_dc"), (3, 5, "bf16_dc")):
        kw = dict(prec=prec, smoother="rbgs" if dim == 2 else "jacobi", omega=1.0 if dim == 2 else 6 / 7,
                  nu=(2, 1) if dim == 2 else (2, 2), inner=2)
        sz, fz_, _ = make_problem(dim, m, 900 + dim, **kw)
        sn, fn, _ = make_problem(dim, m, 910 + dim, **kw)
        rng = np.random.default_rng(7 + dim)
        u0 = np.zeros(fn.shape)
        u0[(slice(1, -1),) * dim] = rng.uniform(-1, 1, (fn.shape[0] - 2,) * dim)
        sn.set_solution(u0)
        B = BatchSolver(4)
        pz, pn = B.add(sz), B.add(sn)
        rho = B.step([pz, pn])
        r0 = [oracle.norm(oracle.residual(np.zeros_like(fz_), fz_)), oracle.norm(oracle.residual(u0, fn))]
        for k, (s, f) in enumerate(((sz, fz_), (sn, fn))):
            r1 = oracle.norm(oracle.residual(s.get_solution(), f))
            assert abs(rho[k] - r1 / r0[k]) <= 1e-5 * r1 / r0[k], (dim, k, rho[k], r1 / r0[k])
        # a single-context solve after the batch step starts from the stepped u
        B.remove(pz)
        u1 = sz.get_solution()
        r_start = oracle.norm(oracle.residual(u1, fz_))
        it, rr, _ = sz.solve(1e-10)
        u2 = sz.get_solution()
        assert oracle.norm(oracle.residual(u2, fz_)) <= 1.01e-10 * r_start
        B.close()


def test_batch_tile_rows_knob():
    """The list launches' rows per chunk (mg_batch_set_tile_rows) is a tuning
    knob: every problem still reaches its tolerance by the oracle's residual,
    a problem gives bit for bit the same solution alone and in a mix under the
    same setting, and invalid values are refused."""
    need_gpu()
    from paper_1406_5369_gb300 import BatchSolver
    import paper_1406_5369_gb300._capi as C
    ms = [7, 9, 8, 10]
    probs = [make_problem(2, m, 500 + i, var=True, inner=2) for i, m in enumerate(ms)]
    B = BatchSolver(8)
    B.set_tile_rows(64)  # before the problems are added: kept
    for p in probs:
        B.add(p[0])
    iters, rel = B.solve(1e-8, maxit=60)
    for i, (s, f, k) in enumerate(probs):
        assert rel[i] <= 1e-8
        faces = oracle.node_faces(k)
        u = s.get_solution()
        assert oracle.norm(oracle.residual(u, f, faces=faces)) / oracle.norm(f) <= 1.01e-8
    s, f, k = make_problem(2, ms[3], 503, var=True, inner=2)
    B1 = BatchSolver(1)
    B1.add(s)
    B1.set_tile_rows(64)
    it1, _ = B1.solve(1e-8, maxit=60)
    assert it1[0] == iters[3]
    assert np.array_equal(s.get_solution(), probs[3][0].get_solution())
    with pytest.raises(C.MGError):
        B1.set_tile_rows(-1)
    B.close()
    B1.close()
