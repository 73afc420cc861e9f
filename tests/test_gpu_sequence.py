"""mg_solve_sequence: a stream of right-hand sides solved on two contexts that
take turns, with each problem's host copies overlapping the other context's
solve. Every solution must be bit-for-bit the one a single context gives for
the same right-hand side (same kernels, same launch sequence), whichever of
the two contexts solved it, and must reach the tolerance by the oracle's
residual; argument errors are refused before any work."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,n,kw", [(2, 513, dict(precision="fp32_dc", inner_cycles=2)),
                                      (2, 257, dict(precision="fp64")),
                                      (3, 65, dict(precision="bf16_dc", smoother="jacobi", omega=6 / 7, nu1=2, nu2=2))])
def test_sequence_equals_one_solve_each(dim, n, kw):
    torch = need_gpu()
    from paper_1406_5369_gb300 import Solver, solve_sequence
    streams = [torch.cuda.Stream() for _ in range(3)]
    a, b = (Solver(dim, n, maxit=40, stream=streams[k].cuda_stream, **kw) for k in range(2))
    fs = [torch.from_numpy(synth.uniform_rhs(dim, n, 900 + i)).pin_memory() for i in range(5)]
    us = [torch.empty_like(fs[0]).pin_memory() for _ in range(5)]
    iters, rel = solve_sequence(a, b, fs, us, 1e-10, streams[2].cuda_stream)
    assert np.all(rel <= 1e-10)
    ref = Solver(dim, n, maxit=40, **kw)
    for i in range(5):
        ref.set_rhs(fs[i])
        ref.set_solution(None)
        it, rr, _ = ref.solve(1e-10)
        u = ref.get_solution()
        assert it == iters[i] and rr == rel[i]
        assert np.array_equal(u, us[i].numpy()), i
        f = fs[i].numpy()
        assert oracle.norm(oracle.residual(u, f)) / oracle.norm(f) <= 1.01e-10


def test_sequence_argument_errors():
    torch = need_gpu()
    from paper_1406_5369_gb300 import MGError, Solver, solve_sequence
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    a = Solver(2, 65, stream=s1.cuda_stream)
    b = Solver(2, 65, stream=s2.cuda_stream)
    c = Solver(2, 129, stream=torch.cuda.Stream().cuda_stream)
    f = [np.zeros((65, 65))]
    u = [np.zeros((65, 65))]
    with pytest.raises(MGError):
        solve_sequence(a, a, f, u, 1e-8, torch.cuda.Stream().cuda_stream)  # one context twice
    with pytest.raises(MGError):
        solve_sequence(a, b, f, u, 1e-8, s1.cuda_stream)  # copy stream shared with a context
    with pytest.raises(MGError):
        solve_sequence(a, c, f, u, 1e-8, torch.cuda.Stream().cuda_stream)  # sizes differ
    it, rel = solve_sequence(a, b, [], [], 1e-8, torch.cuda.Stream().cuda_stream)
    assert len(it) == 0
