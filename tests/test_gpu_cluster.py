"""The V-cycle of the small 2D levels on one thread-block cluster
(cluster_max_n): one inner V-cycle of defect correction from zero is the
oracle's FP64 V-cycle (Algorithm 1: RBGS, full weighting, bilinear
interpolation, exact coarsest solve) up to FP32 rounding, for tops of 129^2
and 257^2 (the whole inner cycle, or the levels below a streamed 513^2
level), any sweep counts including nu1 = 0 or nu2 = 0, a relaxation weight
and 3^2, 5^2 and 9^2 coarsest grids; a full solve with it reaches the
tolerance by the oracle's residual in the same number of outer steps as the
per-level kernels, with the same final error bound."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import error_vs_converged_oracle, need_gpu, rel_err

pytestmark = pytest.mark.gpu

CASES = [
    (129, 2, 1, 1.0, 3),
    (257, 2, 1, 1.0, 3),
    (513, 2, 1, 1.0, 3),
    (257, 1, 1, 1.15, 5),
    (513, 0, 2, 1.0, 3),
    (257, 2, 0, 1.0, 9),
    (129, 3, 2, 0.9, 5),
]


def one_inner_cycle(n, nu1, nu2, omega, coarsest, f, cluster):
    from paper_1406_5369_gb300 import Solver
    s = Solver(2, n, precision="fp32_dc", inner_cycles=1, maxit=1, nu1=nu1, nu2=nu2, omega=omega,
               coarsest_n=coarsest, cluster_max_n=0 if cluster else 1)
    s.set_rhs(f)
    s.solve(1e-30, raise_on_noconv=False)
    u, launches = s.get_solution(), s.kernel_launches()
    s.close()
    return u, launches


@pytest.mark.parametrize("n,nu1,nu2,omega,coarsest", CASES)
def test_one_cluster_cycle_is_the_oracle_vcycle(n, nu1, nu2, omega, coarsest):
    need_gpu()
    f = synth.uniform_rhs(2, n, 0xC1 + n + 7 * nu1 + 3 * nu2)
    # one outer step from zero: u = e, one FP32 inner V-cycle on the defect f
    u_on, l_on = one_inner_cycle(n, nu1, nu2, omega, coarsest, f, True)
    u_off, l_off = one_inner_cycle(n, nu1, nu2, omega, coarsest, f, False)
    H = oracle.Hierarchy(2, n, coarsest_n=coarsest, smoother=oracle.RBGS, omega=omega, nu1=nu1, nu2=nu2)
    H.set_rhs(f)
    H.vcycle()
    want = H.get_u()
    assert l_on < l_off  # the levels from 257^2 (or 129^2) down ran as one launch
    # FP32 arithmetic in the inner cycle: a few ulps of FP32 per operation
    assert rel_err(u_on, want) <= 2e-5, rel_err(u_on, want)
    assert rel_err(u_off, want) <= 2e-5
    assert np.all(u_on[0] == 0) and np.all(u_on[-1] == 0) and np.all(u_on[:, 0] == 0) and np.all(u_on[:, -1] == 0)


@pytest.mark.parametrize("n", [257, 1025])
def test_dc_solve_with_the_cluster_cycle(n):
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    f = synth.uniform_rhs(2, n, 0x5EED0002 ^ n)
    out = {}
    for cluster in (True, False):
        s = Solver(2, n, precision="fp32_dc", inner_cycles=3, maxit=30, cluster_max_n=0 if cluster else 1)
        s.set_rhs(f)
        it, rr, hist = s.solve(1e-10)
        out[cluster] = (it, s.get_solution())
        s.close()
    assert out[True][0] == out[False][0]
    u = out[True][1]
    assert oracle.norm(oracle.residual(u, f)) / oracle.norm(f) <= 1.01e-10
    err, bound, _ = error_vs_converged_oracle(u, f)
    assert err <= bound and err <= 1e-9, (err, bound)
    assert rel_err(u, out[False][1]) <= 2e-9


def test_cluster_cycle_timed_as_one_coarse_launch_per_cycle():
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    n = 513
    f = synth.uniform_rhs(2, n, 5)
    s = Solver(2, n, precision="fp32_dc", inner_cycles=2, maxit=30, join_cycles=False)
    s.set_rhs(f)
    s.set_timing(True)
    it, rr, _ = s.solve(1e-10)
    # level 1 (257^2) takes the whole coarse cycle; nothing launches below it
    assert s.timing("coarse", 1)[1] == 2 * it and s.timing("coarse", 1)[0] > 0
    assert s.timing("pre", 1) == (0.0, 0) and s.timing("pre", 2) == (0.0, 0)
    assert s.timing("coarse", s.levels - 1) == (0.0, 0)
    s.set_timing(False)
    s.close()
