"""The oracle's OpenMP timing build (liboracle_mt.so) against its serial
parity build (liboracle.so), bit for bit.

Only loops whose points are independent run in parallel there (one colour of
a red-black sweep, a Jacobi sweep, the residual, the transfers, fills), and
the norm's pairwise sum keeps its tree; so every number must be identical to
the serial oracle's. The timing build is what the benchmark's CPU baseline
and the full-size error checks run; these cases pin it to the parity oracle
on grids with ragged thread splits (odd interior sizes, several threads).
"""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module", autouse=True)
def four_threads():
    used = oracle.set_threads(4)
    assert used == 4
    yield
    oracle.set_threads(oracle.host_cores())


@pytest.mark.parametrize("dim,n,smoother,omega,nu1,nu2,var", [
    (2, 65, oracle.RBGS, 1.0, 2, 1, False),
    (2, 129, oracle.JACOBI, 0.8, 2, 2, False),
    (2, 65, oracle.RBGS, 1.15, 1, 2, True),
    (3, 33, oracle.JACOBI, 6.0 / 7.0, 2, 2, False),
    (3, 17, oracle.RBGS, 1.0, 2, 1, True),
])
def test_solve_history_and_solution_bitwise(dim, n, smoother, omega, nu1, nu2, var):
    f = synth.uniform_rhs(dim, n, 0x5EED0000 + n)
    k = synth.lognormal_k(dim, n, 0x5EED0100 + n) if var else None
    out = []
    for mt in (False, True):
        H = oracle.Hierarchy(dim, n, knode=k, smoother=smoother, omega=omega, nu1=nu1, nu2=nu2, mt=mt)
        H.set_rhs(f)
        rho = H.solve(1e-30, 6)
        out.append((rho, H.get_u(), H.residual_norm()))
    (r0, u0, n0), (r1, u1, n1) = out
    assert np.array_equal(r0, r1)
    assert np.array_equal(u0, u1)
    assert n0 == n1


def test_defect_correction_bitwise():
    n = 65
    f = synth.uniform_rhs(2, n, 3)
    rs = []
    for mt in (False, True):
        H = oracle.Hierarchy(2, n, mt=mt)
        H.set_rhs(f)
        rs.append((H.dc_solve(1e-12, 20), H.get_u()))
    assert np.array_equal(rs[0][0], rs[1][0]) and np.array_equal(rs[0][1], rs[1][1])


@pytest.mark.parametrize("dim,n", [(2, 1), (2, 9), (2, 257), (3, 19), (3, 7)])
def test_residual_and_norm_bitwise(dim, n):
    # norm over m = (n-2)^dim squares: the task-split pairwise tree (including
    # m <= 8 and m = 0) gives the serial sum exactly
    if n < 3:
        n = 3
    u = synth.uniform(10 + n, (n,) * dim)
    f = synth.uniform(20 + n, (n,) * dim)
    r0, r1 = oracle.residual(u, f), oracle.residual(u, f, mt=True)
    assert np.array_equal(r0, r1)
    assert oracle.norm(r0) == oracle.norm(r0, mt=True)
    big = synth.uniform(5, (1025, 1025)) - 0.5
    assert oracle.norm(big) == oracle.norm(big, mt=True)


def test_threads_follow_the_setting():
    assert oracle.set_threads(2) == 2
    assert oracle.set_threads(4) == 4
    assert oracle.lib(mt=False).or_threads() == 1
