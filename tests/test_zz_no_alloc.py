"""The allocation-free residual norm (mg_residual_norm_noalloc).

Callers that may not allocate device memory (no arena, no context) get the
norm ||f - A u||_2 from caller-owned device arrays, with the reduction's
scratch in a static device array of the library. This file checks, through
the C ABI, that two calls in a row give the same value as the context-based
mg_residual_norm within the FP64 norm tolerance of the other GPU tests, and
that grids above the static limit are refused. It is named to run last, and
it builds every object it needs, so it passes alone or after the others.
"""
import ctypes

import numpy as np
import pytest

import synth
from gpu_util import need_gpu, zero_boundary

pytestmark = pytest.mark.gpu

NORM_RTOL = 1e-12  # FP64 norm tolerance used by the operator tests (10 x 1e-13)


def test_noalloc_norm_matches_context_norm_on_consecutive_calls():
    torch = need_gpu()
    from paper_1406_5369_gb300 import Solver, _capi
    lib = _capi.load()
    stream = torch.cuda.current_stream().cuda_stream
    for dim, n in [(2, 1025), (3, 129)]:
        s = Solver(dim, n)
        for call in range(2):
            u = zero_boundary(synth.uniform(1000 * dim + call, (n,) * dim))
            f = synth.uniform(2000 * dim + call, (n,) * dim)
            s.set_rhs(f)
            s.set_solution(u)
            want = s.residual_norm(0)
            ud = torch.from_numpy(u).cuda()
            fd = torch.from_numpy(f).cuda()
            out = ctypes.c_double(-1.0)
            st = lib.mg_residual_norm_noalloc(dim, n, None, ctypes.c_void_p(ud.data_ptr()),
                                              ctypes.c_void_p(fd.data_ptr()), ctypes.byref(out),
                                              ctypes.c_void_p(stream))
            assert st == _capi.MG_OK, lib.mg_last_error()
            assert abs(out.value - want) <= NORM_RTOL * want, (dim, n, call, out.value, want)
        s.close()


def test_noalloc_norm_result_into_device_memory_and_stencil():
    torch = need_gpu()
    from paper_1406_5369_gb300 import Solver, _capi
    lib = _capi.load()
    n = 257
    st3 = _capi.mg_const_stencil(1.0, 0.25, 1.0)
    s = Solver(2, n, stencil=(1.0, 0.25, 1.0))
    u = zero_boundary(synth.uniform(31, (n, n)))
    f = synth.uniform(32, (n, n))
    s.set_rhs(f)
    s.set_solution(u)
    want = s.residual_norm(0)
    ud, fd = torch.from_numpy(u).cuda(), torch.from_numpy(f).cuda()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    for _ in range(2):
        st = lib.mg_residual_norm_noalloc(2, n, ctypes.byref(st3), ctypes.c_void_p(ud.data_ptr()),
                                          ctypes.c_void_p(fd.data_ptr()),
                                          ctypes.cast(ctypes.c_void_p(out.data_ptr()), ctypes.POINTER(ctypes.c_double)),
                                          None)
        assert st == _capi.MG_OK
        assert abs(float(out.item()) - want) <= NORM_RTOL * want


@pytest.mark.parametrize("dim,n,sten", [(3, 65, (1.0, 0.5, 2.0)), (3, 257, None), (2, 8193, None)])
def test_noalloc_norm_3d_anisotropic_and_largest_grids(dim, n, sten):
    """The cz term of the 3D stencil, and the largest accepted grids: 3D n = 257
    (8,097 partial sums) and 2D n = 8193 (32,761 of the 32,768 slots, so the
    finalize loop reads to the end of the static array, next to the result slot)."""
    torch = need_gpu()
    from paper_1406_5369_gb300 import Solver, _capi
    lib = _capi.load()
    cs = None if sten is None else _capi.mg_const_stencil(*sten)
    s = Solver(dim, n, **({} if sten is None else {"stencil": sten}))
    gen = torch.Generator(device="cuda").manual_seed(77 + n)
    ud = torch.rand((n,) * dim, dtype=torch.float64, device="cuda", generator=gen)
    if dim == 2:
        ud[0, :] = ud[-1, :] = ud[:, 0] = ud[:, -1] = 0
    else:
        ud[0], ud[-1], ud[:, 0], ud[:, -1], ud[:, :, 0], ud[:, :, -1] = 0, 0, 0, 0, 0, 0
    fd = 2 * torch.rand((n,) * dim, dtype=torch.float64, device="cuda", generator=gen) - 1
    s.set_rhs(fd)
    s.set_solution(ud)
    want = s.residual_norm(0)
    for _ in range(2):
        out = ctypes.c_double(-1.0)
        st = lib.mg_residual_norm_noalloc(dim, n, None if cs is None else ctypes.byref(cs),
                                          ctypes.c_void_p(ud.data_ptr()), ctypes.c_void_p(fd.data_ptr()),
                                          ctypes.byref(out), None)
        assert st == _capi.MG_OK, lib.mg_last_error()
        assert lib.mg_last_error() == b""
        assert abs(out.value - want) <= NORM_RTOL * want, (dim, n, out.value, want)
    s.close()


def test_noalloc_norm_rejects_grids_above_the_static_limit():
    torch = need_gpu()
    from paper_1406_5369_gb300 import _capi
    lib = _capi.load()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = ctypes.c_double()
    p = ctypes.c_void_p(buf.data_ptr())
    # 511^3 interior nodes need more partial-sum slots than the static scratch has;
    # the size check runs before any launch, so the small buffer is never read.
    assert lib.mg_residual_norm_noalloc(3, 513, None, p, p, ctypes.byref(out), None) == _capi.MG_EINVAL
    assert b"static scratch" in lib.mg_last_error()
    assert lib.mg_residual_norm_noalloc(2, 2, None, p, p, ctypes.byref(out), None) == _capi.MG_EINVAL
    # coefficients that mg_create refuses are refused here too
    bad = _capi.mg_const_stencil(1.0, -1.0, 1.0)
    assert lib.mg_residual_norm_noalloc(2, 3, ctypes.byref(bad), p, p, ctypes.byref(out), None) == _capi.MG_EINVAL
    assert b"stencil" in lib.mg_last_error()
