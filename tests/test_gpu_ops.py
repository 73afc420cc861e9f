"""Operator-level parity of the CUDA library with the FP64 oracle.

Every C-ABI level operator (mg_smooth, mg_residual, mg_restrict,
mg_prolongate, mg_residual_norm, mg_coarse_solve) runs on seeded random
fields at every level of a hierarchy (so the sizes run from 3 up to grids
that span several thread blocks with a ragged last block), in 2D and 3D,
for the constant and the variable stencil and for the three storage
precisions. Inputs are read back after upload, so reduced-precision cases
compare against the oracle applied to the same rounded inputs.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import OP_TOL, interior, need_gpu, rel_err, zero_boundary

pytestmark = pytest.mark.gpu

FINEST = {2: 257, 3: 65}
PRECISIONS = ["fp64", "fp32_dc", "bf16_dc"]


def make(dim, prec, var, smoother="rbgs", omega=1.0, n=None):
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    n = n or FINEST[dim]
    k = synth.lognormal_k(dim, n, 0x5EED0004) if var else None
    s = Solver(dim, n, k=k, precision=prec, smoother=smoother, omega=omega, nu1=2, nu2=1)
    ref = oracle.Hierarchy(dim, n, knode=k)
    return s, ref


def rand_field(dim, n, seed):
    return zero_boundary(synth.uniform(seed, (n,) * dim))


def upload(s, level, field, a):
    s.set_field(level, field, a)
    return s.get_field(level, field)  # values after rounding to storage


def tol(prec, level, s, var=False):
    # The coarsest level is stored in FP64, but with variable coefficients in a
    # defect-correction context its faces are coarsened from FP32 faces.
    if level == s.levels - 1 and not (var and prec != "fp64"):
        return OP_TOL["fp64"]
    return OP_TOL[prec]


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("var", [False, True])
@pytest.mark.parametrize("smoother,omega", [("rbgs", 1.0), ("jacobi", 0.8)])
def test_smooth(dim, prec, var, smoother, omega):
    s, ref = make(dim, prec, var, smoother, omega)
    for l in range(s.levels):
        nl = s.level_size(l)
        u = upload(s, l, "u", rand_field(dim, nl, 100 + l))
        f = upload(s, l, "f", synth.uniform(200 + l, (nl,) * dim))
        s.smooth(l, 2)
        got = s.get_field(l, "u")
        fn = oracle.rbgs if smoother == "rbgs" else oracle.jacobi
        want = fn(u, f, sweeps=2, omega=omega, faces=ref.faces(l))
        assert rel_err(interior(got), interior(want)) <= tol(prec, l, s, var) * 4, (l, nl)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("var", [False, True])
def test_residual(dim, prec, var):
    s, ref = make(dim, prec, var)
    for l in range(s.levels):
        nl = s.level_size(l)
        u = upload(s, l, "u", rand_field(dim, nl, 300 + l))
        f = upload(s, l, "f", synth.uniform(400 + l, (nl,) * dim))
        s.residual(l)
        got = s.get_field(l, "r")
        want = oracle.residual(u, f, faces=ref.faces(l))
        assert rel_err(interior(got), interior(want)) <= tol(prec, l, s, var), (l, nl)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", PRECISIONS)
def test_restrict(dim, prec):
    s, _ = make(dim, prec, False)
    for l in range(s.levels - 1):
        nl = s.level_size(l)
        r = upload(s, l, "r", rand_field(dim, nl, 500 + l))
        s.restrict(l)
        got = s.get_field(l + 1, "f")
        want = oracle.restrict(r)
        assert rel_err(interior(got), interior(want)) <= tol(prec, l + 1, s) + tol(prec, l, s), (l, nl)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", PRECISIONS)
def test_prolongate(dim, prec):
    s, _ = make(dim, prec, False)
    for l in range(s.levels - 1):
        nl, nc = s.level_size(l), s.level_size(l + 1)
        e = upload(s, l + 1, "u", rand_field(dim, nc, 600 + l))
        u = upload(s, l, "u", rand_field(dim, nl, 700 + l))
        s.prolongate(l)
        got = s.get_field(l, "u")
        want = oracle.prolong_add(e, u)
        assert rel_err(interior(got), interior(want)) <= 2 * tol(prec, l, s), (l, nl)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("var", [False, True])
def test_residual_norm(dim, prec, var):
    s, ref = make(dim, prec, var)
    first = 0 if prec == "fp64" else 1  # DC level 0 norm is the outer problem's
    for l in range(first, s.levels):
        nl = s.level_size(l)
        u = upload(s, l, "u", rand_field(dim, nl, 800 + l))
        f = upload(s, l, "f", synth.uniform(900 + l, (nl,) * dim))
        got = s.residual_norm(l)
        want = oracle.norm(oracle.residual(u, f, faces=ref.faces(l)))
        assert abs(got - want) <= 10 * tol(prec, l, s, var) * want, (l, got, want)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("var", [False, True])
def test_outer_residual_norm(dim, prec, var):
    # Level 0 of a defect-correction context is the FP64 outer problem.
    s, ref = make(dim, prec, var)
    n = s.n
    u = rand_field(dim, n, 11)
    f = synth.uniform(12, (n,) * dim)
    s.set_rhs(f)
    s.set_solution(u)
    got = s.residual_norm(0)
    want = oracle.norm(oracle.residual(u, f, faces=ref.faces(0)))
    assert abs(got - want) <= 1e-13 * want


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("var", [False, True])
def test_coarse_solve(dim, var):
    s, ref = make(dim, "fp64", var)
    l = s.levels - 1
    f = upload(s, l, "f", synth.uniform(13, (3,) * dim))
    s.set_field(l, "u", np.zeros((3,) * dim))
    s.coarse_solve()
    got = s.get_field(l, "u")
    want = oracle.dense_solve(f, faces=ref.faces(l))
    assert rel_err(got, want) <= 1e-14


def test_invalid_level_arguments():
    need_gpu()
    from paper_1406_5369_gb300 import MGError, Solver
    s = Solver(2, 9)
    with pytest.raises(MGError):
        s.restrict(s.levels - 1)
    with pytest.raises(MGError):
        s.smooth(s.levels, 1)
    with pytest.raises(MGError):
        s.prolongate(-1)
    with pytest.raises(ValueError):
        s.set_rhs(np.zeros((8, 8)))


def test_bf16_storage_rounds_to_nearest_even():
    # BF16 fields are written with an integer round-to-nearest-even; compare
    # with torch's CPU float32 -> bfloat16 conversion on values that are
    # exact floats: ties at every exponent, neighbours of ties, subnormals,
    # the overflow edge and random values over the whole range.
    torch = pytest.importorskip("torch")
    need_gpu()
    from paper_1406_5369_gb300 import Solver
    n = 65
    s = Solver(2, n, precision="bf16_dc")
    rng = np.random.default_rng(7)
    bits = rng.integers(0, 2 ** 32, size=n * n, dtype=np.uint64).astype(np.uint32)
    e = np.arange(n * n, dtype=np.uint32) % 254 + 1
    ties = (e << 23) | (rng.integers(0, 2 ** 7, size=n * n, dtype=np.uint32) << 16) | 0x8000
    special = np.array([0x00000001, 0x00008000, 0x00018000, 0x007fffff, 0x7f7fffff, 0x7f7f8000, 0x7f7f7fff,
                        0x80008000, 0x3f808000, 0x3f818000, 0x3f80ffff], dtype=np.uint32)
    pool = np.concatenate([bits[: n * n // 3], ties[: n * n // 3], ties[: n * n // 3] + 1, ties[: n * n // 3] - 1])
    pool = pool[(pool & 0x7f800000) != 0x7f800000]  # finite values only
    vals = np.zeros(n * n, dtype=np.uint32)
    vals[: special.size] = special
    vals[special.size:] = pool[: n * n - special.size]
    a = vals.view(np.float32).astype(np.float64).reshape(n, n)
    got = upload(s, 0, "f", a)
    want = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(got, want)
