"""CDSolver: a Python handle on one mg_cd_ctx (include/mg_cd.h), same names as the C ABI.

Implicit Euler steps of nonlinear complex diffusion (Sec. 4) on an n x n
cell-centred grid with Neumann boundaries. Complex fields are numpy
complex128 arrays or torch complex128 tensors (host or CUDA), C-contiguous,
shape (n, n), x fastest. The device arena is a torch uint8 tensor owned by the
solver; the stream defaults to torch's current stream.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _capi as C
from .solver import _SMOOTHER, default_stream_handle

_FIELDS = {"u": C.MG_CD_U, "f": C.MG_CD_F, "r": C.MG_CD_R, "gx": C.MG_CD_GX, "gy": C.MG_CD_GY}


def _cptr(a, n):
    """Raw pointer of a C-contiguous complex128 (n, n) numpy array or torch tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.complex128 or not a.is_contiguous() or a.numel() != n * n:
                raise ValueError("tensor must be contiguous complex128 with n*n elements")
            return ctypes.c_void_p(a.data_ptr()), a
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=np.complex128)
    if arr.size != n * n:
        raise ValueError(f"array has {arr.size} elements, expected {n * n}")
    return ctypes.c_void_p(arr.ctypes.data), arr


class CDSolver:
    """Complex-diffusion time stepping with cell-centred multigrid on the GPU."""

    def __init__(self, n, *, tau=1e-3, theta=np.pi / 30, kappa=0.1, smoother="rbgs", omega=1.0, nu1=2, nu2=2,
                 maxit=50, stream=None, device="cuda"):
        import torch
        self._lib = C.load()
        self.n = n
        p = C.mg_cd_params()
        self._lib.mg_cd_default_params(ctypes.byref(p))
        p.n = int(n)
        p.tau, p.theta, p.kappa = float(tau), float(theta), float(kappa)
        p.smoother = _SMOOTHER[smoother]
        p.omega = float(omega)
        p.nu1, p.nu2 = int(nu1), int(nu2)
        p.maxit = int(maxit)
        p.stream = default_stream_handle() if stream is None else stream
        self._tstream = torch.cuda.current_stream() if stream is None else torch.cuda.ExternalStream(stream)
        self.params = p
        nbytes = self._lib.mg_cd_workspace_bytes(ctypes.byref(p))
        if nbytes == 0:
            raise C.MGError(C.MG_EINVAL, self._lib.mg_last_error().decode())
        self.workspace_bytes = nbytes
        self.arena = torch.empty(nbytes, dtype=torch.uint8, device=device)
        ctx = ctypes.c_void_p()
        C.check(self._lib.mg_cd_create(ctypes.byref(p), ctypes.c_void_p(self.arena.data_ptr()), nbytes,
                                       ctypes.byref(ctx)))
        self.ctx = ctx
        self.levels = self._lib.mg_cd_num_levels(ctx)

    def close(self):
        if getattr(self, "ctx", None):
            self._lib.mg_cd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def level_size(self, level):
        return self._lib.mg_cd_level_size(self.ctx, level)

    def _sync_if_host(self, keep):
        if isinstance(keep, np.ndarray):
            self._tstream.synchronize()

    def set_field(self, level, field, src):
        p, keep = _cptr(src, self.level_size(level))
        C.check(self._lib.mg_cd_set_field(self.ctx, level, _FIELDS[field], p))
        self._sync_if_host(keep)

    def get_field(self, level, field):
        nl = self.level_size(level)
        out = np.empty((nl, nl), np.complex128)
        C.check(self._lib.mg_cd_get_field(self.ctx, level, _FIELDS[field], ctypes.c_void_p(out.ctypes.data)))
        return out

    def begin_step(self, un):
        p, keep = _cptr(un, self.n)
        C.check(self._lib.mg_cd_begin_step(self.ctx, p))
        self._sync_if_host(keep)

    def smooth(self, level, sweeps):
        C.check(self._lib.mg_cd_smooth(self.ctx, level, sweeps))

    def residual(self, level):
        C.check(self._lib.mg_cd_residual(self.ctx, level))

    def restrict(self, level):
        C.check(self._lib.mg_cd_restrict(self.ctx, level))

    def prolongate(self, level):
        C.check(self._lib.mg_cd_prolongate(self.ctx, level))

    def coarse_solve(self):
        C.check(self._lib.mg_cd_coarse_solve(self.ctx))

    def vcycle(self):
        C.check(self._lib.mg_cd_vcycle(self.ctx))

    def residual_norm(self, level=0):
        out = ctypes.c_double()
        C.check(self._lib.mg_cd_residual_norm(self.ctx, level, ctypes.byref(out)))
        return out.value

    def solve(self, tol, raise_on_noconv=True):
        it, rr = ctypes.c_int(), ctypes.c_double()
        hist = np.zeros(self.params.maxit + 1)
        st = self._lib.mg_cd_solve(self.ctx, float(tol), ctypes.byref(it), ctypes.byref(rr),
                                   ctypes.c_void_p(hist.ctypes.data))
        if st != C.MG_OK and (raise_on_noconv or st != C.MG_ENOCONV):
            C.check(st)
        return it.value, rr.value, hist[:it.value + 1]

    def time_step(self, un, tol, raise_on_noconv=True):
        """One implicit Euler step from un; returns (iterations, relres, history); the
        new state is get_field(0, "u")."""
        self.begin_step(un)
        return self.solve(tol, raise_on_noconv)
