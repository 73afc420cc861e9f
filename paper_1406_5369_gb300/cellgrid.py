"""CCSolver: a Python handle on one mg_cc_ctx (include/mg_cc.h), same names as the C ABI.

Cell-centred grids of n = 2^m cells per dimension with Neumann or Dirichlet
faces, solving sigma u - sum_d c_d d^2u/dx_d^2 = f by V-cycles (cell-centred
restriction, constant interpolation). Inputs may be numpy arrays or torch
tensors (host or CUDA), C-contiguous float64 of shape (n,)*dim with x
fastest. The device arena is a torch uint8 tensor owned by the solver; the
stream defaults to torch's current stream.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _capi as C
from .solver import _FIELD, _SMOOTHER, _ptr, default_stream_handle

_BC = {"neumann": C.MG_CC_NEUMANN, "dirichlet": C.MG_CC_DIRICHLET}


class CCSolver:
    """One cell-centred multigrid context: hierarchy, fields and solve loop on the GPU."""

    def __init__(self, dim, n, *, c=(1.0, 1.0, 1.0), sigma=1.0, bc="neumann", smoother="rbgs", omega=1.0,
                 nu1=2, nu2=1, coarsest_n=1, maxit=50, stream=None, device="cuda"):
        import torch
        self._lib = C.load()
        self.dim, self.n = dim, n
        p = C.mg_cc_params()
        self._lib.mg_cc_default_params(ctypes.byref(p))
        p.dim, p.n = int(dim), int(n)
        for d, v in enumerate((list(c) + [1.0] * 3)[:3]):
            p.c[d] = float(v)
        p.sigma = float(sigma)
        p.bc = _BC[bc]
        p.smoother = _SMOOTHER[smoother]
        p.omega = float(omega)
        p.nu1, p.nu2 = int(nu1), int(nu2)
        p.coarsest_n = int(coarsest_n)
        p.maxit = int(maxit)
        p.stream = default_stream_handle() if stream is None else stream
        self._tstream = torch.cuda.current_stream() if stream is None else torch.cuda.ExternalStream(stream)
        self.params = p
        nbytes = self._lib.mg_cc_workspace_bytes(ctypes.byref(p))
        if nbytes == 0:
            raise C.MGError(C.MG_EINVAL, self._lib.mg_last_error().decode())
        self.workspace_bytes = nbytes
        self.arena = torch.empty(nbytes, dtype=torch.uint8, device=device)
        ctx = ctypes.c_void_p()
        C.check(self._lib.mg_cc_create(ctypes.byref(p), ctypes.c_void_p(self.arena.data_ptr()), nbytes,
                                       ctypes.byref(ctx)))
        self.ctx = ctx
        self.levels = self._lib.mg_cc_num_levels(ctx)

    def close(self):
        if getattr(self, "ctx", None):
            self._lib.mg_cc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def level_size(self, level):
        return self._lib.mg_cc_level_size(self.ctx, level)

    def set_field(self, level, field, src):
        p, keep = _ptr(src, self.dim, self.level_size(level))
        C.check(self._lib.mg_cc_set_field(self.ctx, level, _FIELD[field], p))
        if isinstance(keep, np.ndarray):
            self._tstream.synchronize()

    def get_field(self, level, field):
        nl = self.level_size(level)
        out = np.empty((nl,) * self.dim)
        C.check(self._lib.mg_cc_get_field(self.ctx, level, _FIELD[field], ctypes.c_void_p(out.ctypes.data)))
        return out

    def set_rhs(self, f):
        self.set_field(0, "f", f)

    def set_solution(self, u0=None):
        self.set_field(0, "u", np.zeros((self.n,) * self.dim) if u0 is None else u0)

    def get_solution(self):
        return self.get_field(0, "u")

    # ---- operators (Algorithm 1 steps)
    def smooth(self, level, sweeps):
        C.check(self._lib.mg_cc_smooth(self.ctx, level, sweeps))

    def residual(self, level):
        C.check(self._lib.mg_cc_residual(self.ctx, level))

    def restrict(self, level):
        C.check(self._lib.mg_cc_restrict(self.ctx, level))

    def prolongate(self, level):
        C.check(self._lib.mg_cc_prolongate(self.ctx, level))

    def coarse_solve(self):
        C.check(self._lib.mg_cc_coarse_solve(self.ctx))

    def vcycle(self):
        C.check(self._lib.mg_cc_vcycle(self.ctx))

    def residual_norm(self, level=0):
        out = ctypes.c_double()
        C.check(self._lib.mg_cc_residual_norm(self.ctx, level, ctypes.byref(out)))
        return out.value

    def solve(self, tol, raise_on_noconv=True):
        """Returns (iterations, final relative residual, history rho_0..rho_k)."""
        it = ctypes.c_int()
        rr = ctypes.c_double()
        hist = np.zeros(self.params.maxit + 1)
        st = self._lib.mg_cc_solve(self.ctx, float(tol), ctypes.byref(it), ctypes.byref(rr),
                                   ctypes.c_void_p(hist.ctypes.data))
        if st != C.MG_OK and (raise_on_noconv or st != C.MG_ENOCONV):
            C.check(st)
        return it.value, rr.value, hist[:it.value + 1]
