"""FP64 CPU oracle for the multigrid V-cycle: TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library in
``paper_1406_5369_gb300``) never imports it, and it never imports the
product path; the two share only the seeded input generators in ``synth``.

The arithmetic lives in ``mg_oracle.c`` (node-based grids), ``cc_oracle.c``
(cell-centred grids with Neumann or Dirichlet boundaries) and ``cd_oracle.c``
(implicit Euler steps of complex diffusion on cell-centred grids), plain C, FP64,
natural loop order, built with ``-O2 -ffp-contract=off``; this module compiles
them with gcc on first use and wraps them with ctypes. Arrays are numpy float64 of shape
``(n,)*dim`` with x fastest, as in ``synth``. Local Fourier analysis lives in
``oracle.lfa``.

Parity status of each routine (what pins it is in tests/test_oracle_*.py):
stencil apply, residual, RBGS, Jacobi, full weighting, prolongation, dense
coarse solve, V-cycle, solve loop, defect correction (FP64 inner), face
coefficients and their coarsening are all pinned; so are the cell-centred
operator, smoothers, restriction, constant interpolation, dense solve,
V-cycle and solve loop (tests/test_oracle_cc.py), and the complex-diffusion
diffusivity, face averaging and coarsening, operator, smoothers, transfers,
V-cycle and time step (tests/test_oracle_cd.py). No routine is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "mg_oracle.c"), os.path.join(_HERE, "cc_oracle.c"), os.path.join(_HERE, "cd_oracle.c")]
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SO_MT = os.path.join(_BUILD, "liboracle_mt.so")
_lock = threading.Lock()
_libs = {}

RBGS = 0
JACOBI = 1

_D = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False, mt: bool = False) -> str:
    """Compiles the C sources into oracle/_build/liboracle.so (gcc, FP64, no
    FMA); mt=True builds the timing variant liboracle_mt.so with -fopenmp
    (the same loops, independent ones shared out over the host cores; the
    same numbers bit for bit)."""
    os.makedirs(_BUILD, exist_ok=True)
    so = _SO_MT if mt else _SO
    if force or not os.path.exists(so) or os.path.getmtime(so) < max(os.path.getmtime(x) for x in _SRCS):
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-shared", "-fPIC",
                               *(["-fopenmp"] if mt else []), *_SRCS, "-o", tmp, "-lm"])
        os.replace(tmp, so)
    return so


def lib(mt: bool = False):
    """The serial oracle library (mt=False, the parity oracle) or its OpenMP
    timing build (mt=True)."""
    with _lock:
        if mt not in _libs:
            L = ctypes.CDLL(build(mt=mt))
            vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            sig = {
                "or_apply": (None, [i, i, _D, _D, _D, _D, _D, _D]),
                "or_diag": (None, [i, i, _D, _D, _D, _D, _D]),
                "or_residual": (None, [i, i, _D, _D, _D, _D, _D, _D, _D]),
                "or_rbgs": (None, [i, i, _D, _D, _D, _D, d, i, _D, _D]),
                "or_jacobi": (None, [i, i, _D, _D, _D, _D, d, i, _D, _D]),
                "or_restrict": (None, [i, i, _D, _D]),
                "or_prolong_add": (None, [i, i, _D, _D]),
                "or_node_faces": (None, [i, i, _D, _D, _D, _D, _D]),
                "or_coarsen_faces": (None, [i, i, _D, _D, _D, _D, _D, _D]),
                "or_norm": (d, [i, i, _D]),
                "or_dense_solve": (i, [i, i, _D, _D, _D, _D, _D, _D]),
                "or_create": (vp, [i, i, _D, _D, i, i, d, i, i]),
                "or_destroy": (None, [vp]),
                "or_levels": (i, [vp]),
                "or_level_n": (i, [vp, i]),
                "or_get_faces": (None, [vp, i, _D, _D, _D]),
                "or_set_rhs": (None, [vp, _D]),
                "or_set_u": (None, [vp, _D]),
                "or_get_u": (None, [vp, _D]),
                "or_vcycle": (None, [vp]),
                "or_residual_norm": (d, [vp]),
                "or_solve": (i, [vp, d, i, _D]),
                "or_dc_solve": (i, [vp, d, i, _D]),
                "cc_apply": (None, [i, i, _D, d, i, _D, _D]),
                "cc_diag": (None, [i, i, _D, d, i, _D]),
                "cc_residual": (None, [i, i, _D, d, i, _D, _D, _D]),
                "cc_smooth": (None, [i, i, _D, d, i, i, d, i, _D, _D]),
                "cc_restrict": (None, [i, i, _D, _D]),
                "cc_prolong_add": (None, [i, i, _D, _D]),
                "cc_norm": (d, [i, i, _D]),
                "cc_dense_solve": (i, [i, i, _D, d, i, _D, _D]),
                "cc_create": (vp, [i, i, _D, d, i, i, i, d, i, i]),
                "cc_destroy": (None, [vp]),
                "cc_levels": (i, [vp]),
                "cc_level_n": (i, [vp, i]),
                "cc_set_rhs": (None, [vp, _D]),
                "cc_set_u": (None, [vp, _D]),
                "cc_get_u": (None, [vp, _D]),
                "cc_vcycle": (None, [vp]),
                "cc_residual_norm": (d, [vp]),
                "cc_solve": (i, [vp, d, i, _D]),
                "cd_diffusivity": (None, [i, _D, d, d, _D]),
                "cd_faces": (None, [i, _D, _D, _D]),
                "cd_coarsen_faces": (None, [i, _D, _D, _D, _D]),
                "cd_apply": (None, [i, d, _D, _D, _D, _D]),
                "cd_residual": (None, [i, d, _D, _D, _D, _D, _D]),
                "cd_smooth": (None, [i, d, _D, _D, i, d, i, _D, _D]),
                "cd_restrict": (None, [i, _D, _D]),
                "cd_prolong_add": (None, [i, _D, _D]),
                "cd_norm": (d, [i, _D]),
                "cd_create": (vp, [i, d, d, d, i, d, i, i]),
                "cd_destroy": (None, [vp]),
                "cd_levels": (i, [vp]),
                "cd_get_u": (None, [vp, _D]),
                "cd_get_faces": (None, [vp, i, _D, _D]),
                "cd_begin_step": (None, [vp, _D]),
                "cd_vcycle": (None, [vp]),
                "cd_residual_norm": (d, [vp]),
                "cd_time_step": (i, [vp, _D, d, i, _D]),
                "or_set_threads": (None, [i]),
                "or_threads": (i, []),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _libs[mt] = L
    return _libs[mt]


def set_threads(n: int) -> int:
    """Threads of the OpenMP timing build; returns the count it will use."""
    L = lib(mt=True)
    L.or_set_threads(int(n))
    return int(L.or_threads())


def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _grid(a, dim=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if dim is not None and a.ndim != dim:
        raise ValueError("array rank does not match dim")
    return a


def _c3(c):
    return np.ascontiguousarray(np.array([1.0, 1.0, 1.0] if c is None else list(c) + [1.0] * (3 - len(c)),
                                         dtype=np.float64))


def _faces(faces, dim):
    if faces is None:
        return [None, None, None]
    fs = [_grid(x) for x in faces] + [None] * (3 - len(faces))
    return fs[:3]


# ---------------- stateless level operators ----------------

def apply(u, c=None, faces=None):
    """A u at interior nodes (0 on the boundary)."""
    u = _grid(u)
    dim, n = u.ndim, u.shape[0]
    out = np.empty_like(u)
    c3, fs = _c3(c), _faces(faces, dim)
    lib().or_apply(dim, n, _p(c3), _p(fs[0]), _p(fs[1]), _p(fs[2]), _p(u), _p(out))
    return out


def diag(dim, n, c=None, faces=None):
    out = np.empty((n,) * dim)
    c3, fs = _c3(c), _faces(faces, dim)
    lib().or_diag(dim, n, _p(c3), _p(fs[0]), _p(fs[1]), _p(fs[2]), _p(out))
    return out


def residual(u, f, c=None, faces=None, mt=False):
    u, f = _grid(u), _grid(f)
    dim, n = u.ndim, u.shape[0]
    r = np.empty_like(u)
    c3, fs = _c3(c), _faces(faces, dim)
    lib(mt).or_residual(dim, n, _p(c3), _p(fs[0]), _p(fs[1]), _p(fs[2]), _p(u), _p(f), _p(r))
    return r


def rbgs(u, f, sweeps=1, omega=1.0, c=None, faces=None):
    """Returns u after ``sweeps`` omega red-black Gauss-Seidel sweeps."""
    u, f = _grid(u).copy(), _grid(f)
    dim, n = u.ndim, u.shape[0]
    c3, fs = _c3(c), _faces(faces, dim)
    lib().or_rbgs(dim, n, _p(c3), _p(fs[0]), _p(fs[1]), _p(fs[2]), omega, sweeps, _p(u), _p(f))
    return u


def jacobi(u, f, sweeps=1, omega=0.8, c=None, faces=None):
    u, f = _grid(u).copy(), _grid(f)
    dim, n = u.ndim, u.shape[0]
    c3, fs = _c3(c), _faces(faces, dim)
    lib().or_jacobi(dim, n, _p(c3), _p(fs[0]), _p(fs[1]), _p(fs[2]), omega, sweeps, _p(u), _p(f))
    return u


def restrict(r):
    r = _grid(r)
    dim, nf = r.ndim, r.shape[0]
    nc = (nf - 1) // 2 + 1
    fc = np.empty((nc,) * dim)
    lib().or_restrict(dim, nf, _p(r), _p(fc))
    return fc


def prolong_add(e, u):
    """Returns u + P e (u fine, e coarse)."""
    e, u = _grid(e), _grid(u).copy()
    lib().or_prolong_add(e.ndim, e.shape[0], _p(e), _p(u))
    return u


def node_faces(knode, c=None):
    k = _grid(knode)
    dim, n = k.ndim, k.shape[0]
    out = [np.empty_like(k) for _ in range(dim)] + [None] * (3 - dim)
    lib().or_node_faces(dim, n, _p(_c3(c)), _p(k), _p(out[0]), _p(out[1]), _p(out[2]))
    return out[:dim]


def coarsen_faces(faces):
    dim = len(faces)
    fs = [_grid(x) for x in faces] + [None] * (3 - dim)
    nf = fs[0].shape[0]
    nc = (nf - 1) // 2 + 1
    out = [np.empty((nc,) * dim) for _ in range(dim)] + [None] * (3 - dim)
    lib().or_coarsen_faces(dim, nf, _p(fs[0]), _p(fs[1]), _p(fs[2]), _p(out[0]), _p(out[1]), _p(out[2]))
    return out[:dim]


def norm(r, mt=False):
    r = _grid(r)
    return lib(mt).or_norm(r.ndim, r.shape[0], _p(r))


def dense_solve(f, u_boundary=None, c=None, faces=None):
    """Exact solve of the interior system (Gaussian elimination, partial pivoting)."""
    f = _grid(f)
    dim, n = f.ndim, f.shape[0]
    u = np.zeros_like(f) if u_boundary is None else _grid(u_boundary).copy()
    c3, fs = _c3(c), _faces(faces, dim)
    rc = lib().or_dense_solve(dim, n, _p(c3), _p(fs[0]), _p(fs[1]), _p(fs[2]), _p(u), _p(f))
    if rc != 0:
        raise RuntimeError("singular system")
    return u


# ---------------- hierarchy ----------------

class Hierarchy:
    """A grid hierarchy with V-cycle, solve loop and FP64 defect correction.
    mt=True runs it on the OpenMP timing build (bitwise the same results)."""

    def __init__(self, dim, n, c=None, knode=None, coarsest_n=3, smoother=RBGS, omega=1.0,
                 nu1=2, nu2=1, mt=False):
        self.dim, self.n = dim, n
        self._L = lib(mt)
        self._k = None if knode is None else _grid(knode, dim)
        self._c3 = _c3(c)
        self.h = self._L.or_create(dim, n, _p(self._c3), _p(self._k), coarsest_n, smoother,
                                   float(omega), nu1, nu2)
        if not self.h:
            raise ValueError("invalid hierarchy parameters")
        self.levels = self._L.or_levels(self.h)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self._L.or_destroy(h)
            self.h = None

    def level_n(self, l):
        return self._L.or_level_n(self.h, l)

    def faces(self, l):
        if self._k is None:
            return None
        nl = self.level_n(l)
        out = [np.empty((nl,) * self.dim) for _ in range(self.dim)] + [None] * (3 - self.dim)
        self._L.or_get_faces(self.h, l, _p(out[0]), _p(out[1]), _p(out[2]))
        return out[:self.dim]

    def set_rhs(self, f):
        f = _grid(f, self.dim)
        self._L.or_set_rhs(self.h, _p(f))

    def set_u(self, u):
        u = _grid(u, self.dim)
        self._L.or_set_u(self.h, _p(u))

    def get_u(self):
        u = np.empty((self.n,) * self.dim)
        self._L.or_get_u(self.h, _p(u))
        return u

    def vcycle(self):
        self._L.or_vcycle(self.h)

    def residual_norm(self):
        return self._L.or_residual_norm(self.h)

    def solve(self, tol, maxit):
        """Returns the relative residual history rho[0..k] (rho[0] = 1)."""
        rho = np.zeros(maxit + 1)
        k = self._L.or_solve(self.h, float(tol), int(maxit), _p(rho))
        return rho[:k + 1]

    def dc_solve(self, tol, maxit):
        """Defect correction with an FP64 inner V-cycle; rho[0..k]."""
        rho = np.zeros(maxit + 1)
        k = self._L.or_dc_solve(self.h, float(tol), int(maxit), _p(rho))
        return rho[:k + 1]


# ---------------- cell-centred grids (cc_oracle.c) ----------------
# Arrays are (n,)*dim over the cells, x fastest; bc is "neumann" or "dirichlet"
# (homogeneous, on every face of the unit square/cube).

def _bc(bc):
    if bc not in ("neumann", "dirichlet"):
        raise ValueError("bc must be 'neumann' or 'dirichlet'")
    return 1 if bc == "neumann" else 0


def cc_apply(u, c=None, sigma=0.0, bc="neumann"):
    u = _grid(u)
    out = np.empty_like(u)
    lib().cc_apply(u.ndim, u.shape[0], _p(_c3(c)), float(sigma), _bc(bc), _p(u), _p(out))
    return out


def cc_diag(dim, n, c=None, sigma=0.0, bc="neumann"):
    out = np.empty((n,) * dim)
    lib().cc_diag(dim, n, _p(_c3(c)), float(sigma), _bc(bc), _p(out))
    return out


def cc_residual(u, f, c=None, sigma=0.0, bc="neumann"):
    u, f = _grid(u), _grid(f)
    out = np.empty_like(u)
    lib().cc_residual(u.ndim, u.shape[0], _p(_c3(c)), float(sigma), _bc(bc), _p(u), _p(f), _p(out))
    return out


def cc_smooth(u, f, sweeps, smoother=RBGS, omega=1.0, c=None, sigma=0.0, bc="neumann"):
    u = _grid(u).copy()
    f = _grid(f)
    lib().cc_smooth(u.ndim, u.shape[0], _p(_c3(c)), float(sigma), _bc(bc), int(smoother), float(omega),
                    int(sweeps), _p(u), _p(f))
    return u


def cc_restrict(r):
    r = _grid(r)
    dim, nf = r.ndim, r.shape[0]
    out = np.empty((nf // 2,) * dim)
    lib().cc_restrict(dim, nf, _p(r), _p(out))
    return out


def cc_prolong_add(e, u):
    e = _grid(e)
    u = _grid(u).copy()
    lib().cc_prolong_add(e.ndim, e.shape[0], _p(e), _p(u))
    return u


def cc_norm(r):
    r = _grid(r)
    return lib().cc_norm(r.ndim, r.shape[0], _p(r))


def cc_dense_solve(f, c=None, sigma=0.0, bc="neumann"):
    f = _grid(f)
    u = np.zeros_like(f)
    if lib().cc_dense_solve(f.ndim, f.shape[0], _p(_c3(c)), float(sigma), _bc(bc), _p(f), _p(u)) != 0:
        raise RuntimeError("singular system")
    return u


class CCHierarchy:
    """A cell-centred grid hierarchy n, n/2, ..., coarsest_n with V-cycle and solve loop."""

    def __init__(self, dim, n, c=None, sigma=0.0, bc="neumann", coarsest_n=1, smoother=RBGS, omega=1.0,
                 nu1=2, nu2=1):
        self.dim, self.n = dim, n
        self.h = lib().cc_create(dim, n, _p(_c3(c)), float(sigma), _bc(bc), coarsest_n, smoother, float(omega),
                                 nu1, nu2)
        if not self.h:
            raise ValueError("invalid hierarchy parameters")
        self.levels = lib().cc_levels(self.h)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().cc_destroy(h)
            self.h = None

    def level_n(self, l):
        return lib().cc_level_n(self.h, l)

    def set_rhs(self, f):
        lib().cc_set_rhs(self.h, _p(_grid(f, self.dim)))

    def set_u(self, u):
        lib().cc_set_u(self.h, _p(_grid(u, self.dim)))

    def get_u(self):
        u = np.empty((self.n,) * self.dim)
        lib().cc_get_u(self.h, _p(u))
        return u

    def vcycle(self):
        lib().cc_vcycle(self.h)

    def residual_norm(self):
        return lib().cc_residual_norm(self.h)

    def solve(self, tol, maxit):
        """Returns the relative residual history rho[0..k] (rho[0] = 1)."""
        rho = np.zeros(maxit + 1)
        k = lib().cc_solve(self.h, float(tol), int(maxit), _p(rho))
        return rho[:k + 1]


# ---------------- complex diffusion (cd_oracle.c) ----------------
# Complex arrays are numpy complex128 of shape (n, n), x fastest.

def _cgrid(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _pc(a):
    assert a.dtype == np.complex128 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def cd_diffusivity(u, theta, kappa):
    u = _cgrid(u)
    g = np.empty_like(u)
    lib().cd_diffusivity(u.shape[0], _pc(u), float(theta), float(kappa), _pc(g))
    return g


def cd_faces(g):
    g = _cgrid(g)
    gx, gy = np.empty_like(g), np.empty_like(g)
    lib().cd_faces(g.shape[0], _pc(g), _pc(gx), _pc(gy))
    return gx, gy


def cd_coarsen_faces(gx, gy):
    gx, gy = _cgrid(gx), _cgrid(gy)
    nf = gx.shape[0]
    cx, cy = np.empty((nf // 2, nf // 2), np.complex128), np.empty((nf // 2, nf // 2), np.complex128)
    lib().cd_coarsen_faces(nf, _pc(gx), _pc(gy), _pc(cx), _pc(cy))
    return cx, cy


def cd_apply(u, tau, gx, gy):
    u, gx, gy = _cgrid(u), _cgrid(gx), _cgrid(gy)
    out = np.empty_like(u)
    lib().cd_apply(u.shape[0], float(tau), _pc(gx), _pc(gy), _pc(u), _pc(out))
    return out


def cd_residual(u, f, tau, gx, gy):
    u, f, gx, gy = _cgrid(u), _cgrid(f), _cgrid(gx), _cgrid(gy)
    out = np.empty_like(u)
    lib().cd_residual(u.shape[0], float(tau), _pc(gx), _pc(gy), _pc(u), _pc(f), _pc(out))
    return out


def cd_smooth(u, f, tau, gx, gy, sweeps, smoother=RBGS, omega=1.0):
    u = _cgrid(u).copy()
    f, gx, gy = _cgrid(f), _cgrid(gx), _cgrid(gy)
    lib().cd_smooth(u.shape[0], float(tau), _pc(gx), _pc(gy), int(smoother), float(omega), int(sweeps), _pc(u), _pc(f))
    return u


def cd_restrict(r):
    r = _cgrid(r)
    out = np.empty((r.shape[0] // 2,) * 2, np.complex128)
    lib().cd_restrict(r.shape[0], _pc(r), _pc(out))
    return out


def cd_prolong_add(e, u):
    e = _cgrid(e)
    u = _cgrid(u).copy()
    lib().cd_prolong_add(e.shape[0], _pc(e), _pc(u))
    return u


def cd_norm(r):
    r = _cgrid(r)
    return lib().cd_norm(r.shape[0], _pc(r))


class CDHierarchy:
    """Implicit Euler steps of complex diffusion on an n x n cell-centred grid."""

    def __init__(self, n, tau, theta, kappa, smoother=RBGS, omega=1.0, nu1=2, nu2=2):
        self.n = n
        self.h = lib().cd_create(n, float(tau), float(theta), float(kappa), smoother, float(omega), nu1, nu2)
        if not self.h:
            raise ValueError("invalid parameters")
        self.levels = lib().cd_levels(self.h)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().cd_destroy(h)
            self.h = None

    def begin_step(self, un):
        un = _cgrid(un)
        lib().cd_begin_step(self.h, _pc(un))

    def faces(self, l):
        nl = self.n >> l
        gx, gy = np.empty((nl, nl), np.complex128), np.empty((nl, nl), np.complex128)
        lib().cd_get_faces(self.h, l, _pc(gx), _pc(gy))
        return gx, gy

    def vcycle(self):
        lib().cd_vcycle(self.h)

    def residual_norm(self):
        return lib().cd_residual_norm(self.h)

    def get_u(self):
        u = np.empty((self.n, self.n), np.complex128)
        lib().cd_get_u(self.h, _pc(u))
        return u

    def time_step(self, un, tol, maxit):
        """Solves one step from un; returns (u^{n+1}, rho history)."""
        un = _cgrid(un)
        rho = np.zeros(maxit + 1)
        k = lib().cd_time_step(self.h, _pc(un), float(tol), int(maxit), rho.ctypes.data_as(_D))
        return self.get_u(), rho[:k + 1]
