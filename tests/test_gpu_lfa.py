"""The LFA-chosen relaxation weight on the GPU (autotune.lfa_choice).

For the 2D Poisson V(2,1) red-black cycle, LFA picks an over-relaxed weight
(omega ~ 1.15, two-grid factor ~ 0.018 against 0.053 at omega = 1). On the
GPU the FP64 V-cycles with that weight must (1) match the oracle cycle by
cycle (1e-12), (2) contract at close to the predicted factor and (3) reach
1e-10 in fewer cycles than omega = 1; FP32 defect correction with it must
still reach 1e-10.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def test_lfa_omega_on_the_gpu():
    need_gpu()
    from paper_1406_5369_gb300 import Solver, autotune
    choice = autotune.lfa_choice(2, smoothers=("rbgs",), nus=[(2, 1)])
    om = choice["omega"]
    n = 1025
    f = synth.uniform_rhs(2, n, 0x5EED00F3)
    its = {}
    for w in (1.0, om):
        s = Solver(2, n, omega=w, maxit=30)
        s.set_rhs(f)
        it, rr, hist = s.solve(1e-10)
        its[w] = it
        if w == om:
            q = (hist[it] / hist[it - 3]) ** (1 / 3)
            assert q <= 1.3 * choice["rho"] + 0.005, (q, choice["rho"])
            ref = oracle.Hierarchy(2, n, omega=w)
            ref.set_rhs(f)
            rho = ref.solve(0.0, it)
            assert np.max(np.abs(hist - rho)) <= 1e-12
    assert its[om] < its[1.0], its
    s = Solver(2, n, omega=om, precision="fp32_dc", inner_cycles=2, maxit=20)
    s.set_rhs(f)
    _, rr, _ = s.solve(1e-10)
    assert rr <= 1e-10
