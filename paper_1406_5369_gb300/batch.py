"""BatchSolver: many independent problems stepped together (mg_batch_* in mg.h).

Each problem is a Solver (its own arena, right-hand side, solution and
tolerance); the batch steps all of them with level-grouped launches. Only
argument marshalling happens here.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _capi as C
from .solver import default_stream_handle


class BatchSolver:
    def __init__(self, max_problems, stream=None, device="cuda"):
        import torch
        self._lib = C.load()
        nbytes = self._lib.mg_batch_workspace_bytes(int(max_problems))
        if nbytes == 0:
            raise C.MGError(C.MG_EINVAL, "max_problems must be positive")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        h = ctypes.c_void_p()
        st = default_stream_handle() if stream is None else stream
        C.check(self._lib.mg_batch_create(int(max_problems), ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                          st, ctypes.byref(h)))
        self.h = h
        self.max_problems = int(max_problems)
        self.members = {}

    def add(self, solver):
        i = ctypes.c_int()
        C.check(self._lib.mg_batch_add(self.h, solver.ctx, ctypes.byref(i)))
        self.members[i.value] = solver
        return i.value

    def remove(self, pid):
        C.check(self._lib.mg_batch_remove(self.h, int(pid)))
        self.members.pop(pid, None)

    def step(self, ids):
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        rho = np.zeros(len(ids))
        C.check(self._lib.mg_batch_step(self.h, ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(ids),
                                        rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return rho

    def step_async(self, ids):
        """Enqueues one step (mg_batch_step_async); step_wait() completes it."""
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        self._pending = len(ids)
        C.check(self._lib.mg_batch_step_async(self.h, ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(ids)))

    def step_wait(self):
        """Waits for the step in flight; returns rho in the order of its ids."""
        rho = np.zeros(max(getattr(self, "_pending", 0), 1))
        C.check(self._lib.mg_batch_step_wait(self.h, rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return rho[: self._pending]

    def solve(self, tol, maxit=50, raise_on_noconv=True):
        """tol: scalar or {id: tol}; returns (iters, relres) arrays indexed by id."""
        tols = np.zeros(self.max_problems)
        for pid in self.members:
            tols[pid] = tol[pid] if isinstance(tol, dict) else float(tol)
        iters = np.zeros(self.max_problems, dtype=np.int32)
        rel = np.zeros(self.max_problems)
        st = self._lib.mg_batch_solve(self.h, tols.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(maxit),
                                      iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                      rel.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if st != C.MG_OK and (raise_on_noconv or st != C.MG_ENOCONV):
            C.check(st)
        return iters, rel

    def set_inner_cycles(self, n):
        C.check(self._lib.mg_batch_set_inner_cycles(self.h, int(n)))

    def set_tile_rows(self, rows):
        """Rows per warp chunk of the fused 2D list launches (0 = 256)."""
        C.check(self._lib.mg_batch_set_tile_rows(self.h, int(rows)))

    def set_capture(self, on):
        """True (default): solve() replays captured steps with the stopping
        test on the device; False: one mg_batch_step per step."""
        C.check(self._lib.mg_batch_set_capture(self.h, 1 if on else 0))

    def launches(self):
        return self._lib.mg_batch_launches(self.h)

    KINDS = {"pre": 0, "post": 1, "coarse": 2, "outer": 3, "update": 4, "norm": 5}

    def set_timing(self, on):
        """CUDA-event timing of the launch groups of uncaptured steps."""
        C.check(self._lib.mg_batch_set_timing(self.h, 1 if on else 0))

    def timing(self, kind):
        """(total ms, timed launch groups, algorithmic bytes) of one kernel kind."""
        ms, n, by = ctypes.c_double(), ctypes.c_ulonglong(), ctypes.c_double()
        C.check(self._lib.mg_batch_get_timing(self.h, self.KINDS[kind], ctypes.byref(ms), ctypes.byref(n),
                                              ctypes.byref(by)))
        return ms.value, n.value, by.value

    def reset_timing(self):
        C.check(self._lib.mg_batch_reset_timing(self.h))

    def solve_profile(self):
        """Host milliseconds of the last captured solve's phases (set-up,
        capture + instantiate, replays), replays launched, kernels per replay."""
        out = (ctypes.c_double * 5)()
        C.check(self._lib.mg_batch_solve_profile(self.h, out))
        return {"setup_ms": out[0], "capture_ms": out[1], "replays_ms": out[2], "replays": int(out[3]),
                "kernels_per_replay": int(out[4])}

    def close(self):
        if getattr(self, "h", None):
            self._lib.mg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
