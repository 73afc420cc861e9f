"""Arena guard zones (options.canary): every buffer of a context is followed
by 256 bytes of 0xA5 that no kernel or copy may touch. After full solves of
every kernel family - FP64 per-level kernels, the packed FP32 fused 2D
kernels with constant and variable stencils, the cluster and single-block
coarse cycles, the exact outer step, Jacobi, 3D BF16 defect correction, dense
coarsest inverses and the batch engine's list launches - every zone is intact,
and the solution is bit for bit the one of the same solver without zones.
A zone changed from the host is reported with the buffer it follows."""
import numpy as np
import pytest

import synth
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

CASES = [
    dict(dim=2, n=129, precision="fp64"),
    dict(dim=2, n=129, precision="fp64", coarsest_n=9, use_graph=False),
    dict(dim=2, n=1025, precision="fp32_dc", inner_cycles=2),
    dict(dim=2, n=513, precision="fp32_dc", var=True),
    dict(dim=2, n=257, precision="bf16_dc", smoother="jacobi", omega=0.8),
    dict(dim=3, n=33, precision="fp64", coarsest_n=5),
    dict(dim=3, n=65, precision="bf16_dc", smoother="jacobi", omega=6 / 7, nu1=2, nu2=2),
    dict(dim=3, n=33, precision="fp32_dc", var=True, coarsest_n=5),
]


def _solve(case, canary, seed):
    from paper_1406_5369_gb300 import Solver
    kw = dict(case)
    dim, n, var = kw.pop("dim"), kw.pop("n"), kw.pop("var", False)
    k = synth.lognormal_k(dim, n, seed ^ 0x77) if var else None
    s = Solver(dim, n, k=k, maxit=40, canary=canary, **kw)
    s.set_rhs(synth.uniform_rhs(dim, n, seed))
    s.solve(1e-9, raise_on_noconv=False)
    u = s.get_solution()
    return s, u


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(f"{v}" for v in c.values()))
def test_solves_leave_every_guard_zone_intact(case):
    need_gpu()
    seed = 0xCA0 + case["n"] + 10 * case["dim"]
    s, u = _solve(case, True, seed)
    # the per-level access path writes and reads fields too
    if s.levels > 1:
        g = s.get_field(1, "f")
        s.set_field(1, "f", g)
    damaged, msg = s.check_canaries()
    s.close()
    assert damaged == 0, msg
    t, u_plain = _solve(case, False, seed)
    t.close()
    assert np.array_equal(u, u_plain)


def test_batch_steps_leave_every_guard_zone_intact():
    need_gpu()
    from paper_1406_5369_gb300 import BatchSolver, Solver
    # one batch per option set (a batch holds problems of one dimension,
    # smoother, relaxation weight, sweep counts and precision)
    groups = [
        (2, [65, 257, 129], dict(precision="fp32_dc"), True),
        (2, [65, 513], dict(precision="fp32_dc"), False),
        (3, [17, 33], dict(precision="bf16_dc", smoother="jacobi", omega=6 / 7, nu1=2, nu2=2), False),
    ]
    for g, (dim, sizes, kw, var) in enumerate(groups):
        solvers = []
        for i, n in enumerate(sizes):
            k = synth.lognormal_k(dim, n, 0xBA7 + i) if var else None
            s = Solver(dim, n, k=k, maxit=60, canary=True, **kw)
            s.set_rhs(synth.uniform_rhs(dim, n, 0xBA0 + 16 * g + i))
            solvers.append(s)
        B = BatchSolver(len(solvers))
        for s in solvers:
            B.add(s)
        B.solve(1e-8, raise_on_noconv=False)
        B.close()
        for s in solvers:
            damaged, msg = s.check_canaries()
            s.close()
            assert damaged == 0, (g, msg)


def test_a_changed_zone_is_reported_with_its_buffer():
    need_gpu()
    import torch
    from paper_1406_5369_gb300 import Solver
    from paper_1406_5369_gb300._capi import MGError
    n = 129
    s = Solver(2, n, canary=True)
    # FP64 rows are padded to 128 bytes (16 values): the finest u[0] holds
    # 144 x 129 values from offset 0, its zone follows at once, and u[1]
    # starts at the next 256-byte boundary after that zone.
    u_bytes = 144 * n * 8
    zone_u0 = u_bytes
    zone_u1 = (u_bytes + 256 + 255) // 256 * 256 + u_bytes
    assert s.check_canaries() == (0, "")
    s.arena[zone_u0] = 0
    torch.cuda.synchronize()
    damaged, msg = s.check_canaries()
    assert damaged == 1 and "after l0.u0, byte 0 " in msg, msg
    s.arena[zone_u0] = 0xA5
    s.arena[zone_u1 + 17] = 1
    s.arena[zone_u1 + 255] = 1
    torch.cuda.synchronize()
    damaged, msg = s.check_canaries()
    assert damaged == 1 and "after l0.u1, byte 17 " in msg, msg
    s.close()
    t = Solver(2, n)
    with pytest.raises(MGError):
        t.check_canaries()
    t.close()
