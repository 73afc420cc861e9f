"""Small driver for kernel profilers: a few warm solves of one seeded Poisson
problem, then one more solve.

    python -m paper_1406_5369_gb300.profile_solve --dim 2 --n 4097 --precision fp32_dc

Every solve repeats the same launch sequence. The right-hand side is drawn on
the host (i.i.d. U[-1, 1] at interior nodes, synth.uniform_rhs) and copied,
so every kernel the process launches is the library's; the script prints
how many ran before the last solve and how many the last solve took, which
are the -s/-c arguments that select that solve in a profiler's launch list.
"""
from __future__ import annotations

import argparse
import os
import sys


def main(argv=None) -> int:
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import synth
    from paper_1406_5369_gb300 import Solver

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--dim", type=int, default=2)
    ap.add_argument("--n", type=int, default=4097)
    ap.add_argument("--precision", default="fp32_dc", choices=["fp64", "fp32_dc", "bf16_dc"])
    ap.add_argument("--smoother", default="rbgs", choices=["rbgs", "jacobi"])
    ap.add_argument("--omega", type=float, default=1.0)
    ap.add_argument("--nu1", type=int, default=2)
    ap.add_argument("--nu2", type=int, default=1)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--warm", type=int, default=2)
    ap.add_argument("--inner-cycles", type=int, default=1)
    ap.add_argument("--lognormal-k", action="store_true",
                    help="variable coefficient k = exp(N(0,1)) per node (synth.lognormal_k)")
    a = ap.parse_args(argv)
    f = torch.from_numpy(synth.uniform_rhs(a.dim, a.n, synth.WORKLOAD_SEED_BASE + 2)).cuda()
    k = synth.lognormal_k(a.dim, a.n, synth.WORKLOAD_SEED_BASE + 4) if a.lognormal_k else None
    s = Solver(a.dim, a.n, k=k, precision=a.precision, smoother=a.smoother, omega=a.omega, nu1=a.nu1, nu2=a.nu2,
               inner_cycles=a.inner_cycles, maxit=80)
    s.set_rhs(f)
    for _ in range(a.warm):
        s.set_solution(None)
        s.solve(a.tol)
    torch.cuda.synchronize()
    before = s.kernel_launches()
    s.set_solution(None)
    it, rel, _ = s.solve(a.tol)
    torch.cuda.synchronize()
    print(f"dim={a.dim} n={a.n} precision={a.precision} smoother={a.smoother} cycles={it} relres={rel:.3e} "
          f"launches_before_last_solve={before} launches_last_solve={s.kernel_launches() - before}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
