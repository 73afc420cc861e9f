"""Solver: a Python handle on one mg_ctx (include/mg.h), same names as the C ABI.

Inputs may be numpy arrays (host memory) or torch tensors (host or CUDA);
they are passed to the library as raw pointers and must be C-contiguous
float64 of shape (n,)*dim with x fastest. The device arena is a torch uint8
tensor owned by the Solver; the stream defaults to torch's current stream.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _capi as C

_PRECISION = {"fp64": C.MG_FP64, "fp32_dc": C.MG_FP32_DC, "bf16_dc": C.MG_BF16_DC}
_SMOOTHER = {"rbgs": C.MG_RBGS, "jacobi": C.MG_JACOBI}
_FIELD = {"u": C.MG_FIELD_U, "f": C.MG_FIELD_F, "r": C.MG_FIELD_R}


def _ptr(a, dim=None, n=None):
    """Raw pointer of a C-contiguous float64 numpy array or torch tensor."""
    if a is None:
        return None, None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64 or not a.is_contiguous():
                raise ValueError("tensor must be contiguous float64")
            if n is not None and a.numel() != n ** dim:
                raise ValueError("tensor has the wrong number of elements")
            return ctypes.c_void_p(a.data_ptr()), a
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and arr.size != n ** dim:
        raise ValueError(f"array has {arr.size} elements, expected {n ** dim}")
    return ctypes.c_void_p(arr.ctypes.data), arr


def default_stream_handle():
    import torch
    return torch.cuda.current_stream().cuda_stream


class Solver:
    """One multigrid context: hierarchy, fields and solve loop on the GPU."""

    def __init__(self, dim, n, *, stencil=(1.0, 1.0, 1.0), k=None, dirichlet=None,
                 smoother="rbgs", omega=1.0, nu1=2, nu2=1, maxit=50, precision="fp64",
                 fuse=True, use_graph=True, inner_cycles=1, exact_outer=True, tile_rows=0, tile_max_n=0,
                 fuse_depth=0, join_cycles=True, cluster_max_n=0, coarsest_n=3, stream=None, device="cuda", arena=None,
                 canary=False):
        import torch
        self._lib = C.load()
        self.dim, self.n = dim, n
        opt = C.mg_options()
        self._lib.mg_default_options(ctypes.byref(opt))
        opt.smoother = _SMOOTHER[smoother]
        opt.omega = float(omega)
        opt.nu1, opt.nu2 = int(nu1), int(nu2)
        opt.coarsest_n = int(coarsest_n)
        opt.maxit = int(maxit)
        opt.precision = _PRECISION[precision]
        opt.fuse = int(bool(fuse))
        opt.use_graph = int(bool(use_graph))
        opt.inner_cycles = int(inner_cycles)
        opt.exact_outer = int(bool(exact_outer))
        opt.tile_rows = int(tile_rows)
        opt.tile_max_n = int(tile_max_n)
        opt.fuse_depth = int(fuse_depth)
        opt.join_cycles = int(bool(join_cycles))
        opt.cluster_max_n = int(cluster_max_n)
        opt.canary = int(bool(canary))
        opt.stream = default_stream_handle() if stream is None else stream
        self._tstream = torch.cuda.current_stream() if stream is None else torch.cuda.ExternalStream(stream)
        self.opt = opt
        nbytes = self._lib.mg_workspace_bytes(dim, n, int(k is not None), ctypes.byref(opt))
        if nbytes == 0:
            raise C.MGError(C.MG_EINVAL, self._lib.mg_last_error().decode())
        self.workspace_bytes = nbytes
        if arena is None:
            self.arena = torch.empty(nbytes, dtype=torch.uint8, device=device)
        else:
            # the caller's device memory (a uint8 tensor of at least nbytes,
            # 256-byte aligned), e.g. a slice of a pool it manages itself
            if arena.numel() < nbytes or arena.data_ptr() % 256:
                raise ValueError("arena must hold workspace_bytes and start 256-byte aligned")
            self.arena = arena
        st = C.mg_const_stencil(*[float(x) for x in (list(stencil) + [1.0] * 3)[:3]])
        kp, self._k_keep = _ptr(k, dim, n)
        bc = None
        if dirichlet is not None:
            dp, self._bc_keep = _ptr(dirichlet, dim, n)
            bc = C.mg_boundary(0, dp)
        ctx = ctypes.c_void_p()
        C.check(self._lib.mg_create(dim, n, ctypes.byref(st), kp, ctypes.byref(bc) if bc else None,
                                    ctypes.byref(opt), ctypes.c_void_p(self.arena.data_ptr()),
                                    nbytes, ctypes.byref(ctx)))
        self.ctx = ctx
        self._k_keep = None
        self._bc_keep = None
        self.levels = self._lib.mg_num_levels(ctx)

    def close(self):
        if getattr(self, "ctx", None):
            self._lib.mg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check_canaries(self):
        """Debug check of a solver built with canary=True: (number of damaged
        guard zones, message naming the first). A zone is damaged when a
        kernel or copy wrote past the end of the arena buffer before it."""
        bad = ctypes.c_int()
        C.check(self._lib.mg_check_canaries(self.ctx, ctypes.byref(bad)))
        return bad.value, (self._lib.mg_last_error().decode() if bad.value else "")

    def kernel_launches(self):
        return self._lib.mg_kernel_launches(self.ctx)

    def set_timing(self, on=True, level0_only=False, outer_only=False):
        """CUDA-event timing of every kernel (on=True), of level-0 kernels only
        (level0_only=True), of the outer step of defect correction only
        (outer_only=True), or off."""
        C.check(self._lib.mg_set_timing(self.ctx, (3 if outer_only else 2 if level0_only else 1) if on else 0))

    def reset_timing(self):
        C.check(self._lib.mg_reset_timing(self.ctx))

    def timing(self, kind, level=0):
        """(total milliseconds, launches) of one kernel class on one level."""
        kinds = {"pre": C.MG_KERNEL_PRESMOOTH, "post": C.MG_KERNEL_POSTSMOOTH, "coarse": C.MG_KERNEL_COARSE,
                 "outer": C.MG_KERNEL_OUTER, "norm": C.MG_KERNEL_NORM, "other": C.MG_KERNEL_OTHER,
                 "postpre": C.MG_KERNEL_POSTPRE}
        ms = ctypes.c_double()
        cnt = ctypes.c_ulonglong()
        C.check(self._lib.mg_get_timing(self.ctx, kinds.get(kind, kind), level, ctypes.byref(ms), ctypes.byref(cnt)))
        return ms.value, cnt.value

    def level_size(self, level):
        return self._lib.mg_level_size(self.ctx, level)

    # ---- finest-level data
    def set_rhs(self, f):
        p, keep = _ptr(f, self.dim, self.n)
        C.check(self._lib.mg_set_rhs(self.ctx, p))
        self._sync_if_host(keep)

    def set_solution(self, u0=None):
        p, keep = _ptr(u0, self.dim, self.n)
        C.check(self._lib.mg_set_solution(self.ctx, p))
        self._sync_if_host(keep)

    def get_solution(self, out=None):
        if out is None:
            out = np.empty((self.n,) * self.dim)
        p, _ = _ptr(out, self.dim, self.n)
        C.check(self._lib.mg_get_solution(self.ctx, p))
        return out

    def set_field(self, level, field, src):
        nl = self.level_size(level)
        p, keep = _ptr(src, self.dim, nl)
        C.check(self._lib.mg_set_field(self.ctx, level, _FIELD[field], p))
        self._sync_if_host(keep)

    def get_field(self, level, field):
        nl = self.level_size(level)
        out = np.empty((nl,) * self.dim)
        C.check(self._lib.mg_get_field(self.ctx, level, _FIELD[field], ctypes.c_void_p(out.ctypes.data)))
        return out

    def _sync_if_host(self, keep):
        # Host-memory sources are read by asynchronous copies; keep them alive
        # until the stream has consumed them.
        if isinstance(keep, np.ndarray):
            self._tstream.synchronize()

    # ---- operators (Algorithm 1 steps)
    def smooth(self, level, sweeps):
        C.check(self._lib.mg_smooth(self.ctx, level, sweeps))

    def residual(self, level):
        C.check(self._lib.mg_residual(self.ctx, level))

    def restrict(self, level):
        C.check(self._lib.mg_restrict(self.ctx, level))

    def prolongate(self, level):
        C.check(self._lib.mg_prolongate(self.ctx, level))

    def coarse_solve(self):
        C.check(self._lib.mg_coarse_solve(self.ctx))

    def vcycle(self):
        C.check(self._lib.mg_vcycle(self.ctx))

    def residual_norm(self, level=0):
        out = ctypes.c_double()
        C.check(self._lib.mg_residual_norm(self.ctx, level, ctypes.byref(out)))
        return out.value

    def solve(self, tol, raise_on_noconv=True):
        """Returns (iterations, final relative residual, history rho_0..rho_k)."""
        it = ctypes.c_int()
        rr = ctypes.c_double()
        hist = np.zeros(self.opt.maxit + 1)
        st = self._lib.mg_solve(self.ctx, float(tol), ctypes.byref(it), ctypes.byref(rr),
                                ctypes.c_void_p(hist.ctypes.data))
        if st != C.MG_OK and (raise_on_noconv or st != C.MG_ENOCONV):
            C.check(st)
        return it.value, rr.value, hist[:it.value + 1]


def solve_sequence(a, b, fs, us, tol, copy_stream):
    """Solves right-hand sides fs[i] into us[i] (mg_solve_sequence): Solvers
    a and b (same problem settings, each on its own stream) take the
    problems in turn, and each problem's host copies run on `copy_stream`
    (a third stream handle) beside the other Solver's solve. fs / us: float64
    arrays or tensors of n^dim elements, host (pinned for overlap) or device.
    Returns (iters, relres) as numpy arrays."""
    lib = C.load()
    count = len(fs)
    if len(us) != count:
        raise ValueError("fs and us differ in length")
    keep = []
    fp = (ctypes.c_void_p * max(count, 1))()
    up = (ctypes.c_void_p * max(count, 1))()
    for i in range(count):
        p, k = _ptr(fs[i], a.dim, a.n)
        q, k2 = _ptr(us[i], a.dim, a.n)
        fp[i], up[i] = p, q
        keep += [k, k2]
    iters = np.zeros(max(count, 1), dtype=np.int32)
    rel = np.zeros(max(count, 1))
    C.check(lib.mg_solve_sequence(a.ctx, b.ctx, ctypes.c_void_p(copy_stream), count, fp, up, float(tol),
                                  iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  rel.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return iters[:count], rel[:count]
