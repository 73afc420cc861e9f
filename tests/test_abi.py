"""Host-side checks of the C ABI: the library builds, loads and exports every
function include/mg.h declares; argument validation needs no GPU; the product
package never reaches the oracle."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1406_5369_gb300 import build as b
    b.build()
    from paper_1406_5369_gb300 import _capi
    return _capi.load()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_every_declared_function_is_exported(lib):
    from paper_1406_5369_gb300 import _capi
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
        assert name in _capi.SIGNATURES, f"binding lacks {name}"


def test_binding_declares_only_header_functions():
    from paper_1406_5369_gb300 import _capi
    assert set(_capi.SIGNATURES) <= set(declared_functions())


def test_default_options_and_workspace(lib):
    from paper_1406_5369_gb300 import _capi as C
    o = C.mg_options()
    lib.mg_default_options(ctypes.byref(o))
    assert (o.smoother, o.omega, o.nu1, o.nu2, o.coarsest_n, o.precision) == (C.MG_RBGS, 1.0, 2, 1, 3, C.MG_FP64)
    b129 = lib.mg_workspace_bytes(2, 129, 0, ctypes.byref(o))
    # four FP64 fields per level, rows padded to 16 doubles: 129 -> 144, ...
    assert b129 >= 4 * 144 * 129 * 8
    assert lib.mg_workspace_bytes(2, 129, 1, ctypes.byref(o)) > b129
    assert lib.mg_workspace_bytes(2, 100, 0, ctypes.byref(o)) == 0
    assert lib.mg_workspace_bytes(4, 129, 0, ctypes.byref(o)) == 0
    o.precision = C.MG_FP32_DC
    dc = lib.mg_workspace_bytes(2, 8193, 0, ctypes.byref(o))
    o.precision = C.MG_FP64
    fp = lib.mg_workspace_bytes(2, 8193, 0, ctypes.byref(o))
    # outer FP64 u, f, staging plus the FP32 inner hierarchy
    assert fp < dc < 2 * fp


@pytest.mark.parametrize("dim,n,variable,precision,coarsest", [
    (2, 129, 0, "MG_FP64", 3), (2, 129, 1, "MG_FP32_DC", 5), (3, 33, 1, "MG_BF16_DC", 9), (3, 65, 0, "MG_FP64", 3)])
def test_canary_layout_adds_one_guard_zone_per_buffer(lib, dim, n, variable, precision, coarsest):
    """options.canary = 1 puts a 256-byte guard zone after every arena buffer:
    four fields per level (plus dim face arrays with variable k), the dense
    coarsest inverse when the coarsest grid is above 3, the outer FP64 level of
    defect correction (four fields plus faces), and the norm partials, the norm
    result and the scale words. Each zone adds exactly 256 bytes, since every
    buffer starts 256-byte aligned."""
    from paper_1406_5369_gb300 import _capi as C
    o = C.mg_options()
    lib.mg_default_options(ctypes.byref(o))
    assert o.canary == 0
    o.precision = getattr(C, precision)
    o.coarsest_n = coarsest
    plain = lib.mg_workspace_bytes(dim, n, variable, ctypes.byref(o))
    o.canary = 1
    guarded = lib.mg_workspace_bytes(dim, n, variable, ctypes.byref(o))
    levels, m = 0, n
    while m >= coarsest:
        levels += 1
        if m == coarsest:
            break
        m = (m - 1) // 2 + 1
    per_level = 4 + (dim if variable else 0)
    zones = levels * per_level + (1 if coarsest > 3 else 0) + 3
    if precision != "MG_FP64":
        zones += 4 + (dim if variable else 0)
    assert plain > 0 and guarded - plain == 256 * zones
    o.canary = 2
    assert lib.mg_workspace_bytes(dim, n, variable, ctypes.byref(o)) == 0


def test_invalid_arguments_are_rejected_before_any_device_work(lib):
    from paper_1406_5369_gb300 import _capi as C
    o = C.mg_options()
    lib.mg_default_options(ctypes.byref(o))
    ctx = ctypes.c_void_p()
    buf = ctypes.c_void_p(256)
    assert lib.mg_create(2, 10, None, None, None, ctypes.byref(o), buf, 1 << 20, ctypes.byref(ctx)) == C.MG_EINVAL
    assert b"2^m+1" in lib.mg_last_error()
    o.omega = 2.5
    assert lib.mg_create(2, 9, None, None, None, ctypes.byref(o), buf, 1 << 20, ctypes.byref(ctx)) == C.MG_EINVAL
    lib.mg_default_options(ctypes.byref(o))
    o.coarsest_n = 7  # not of the form 2^m+1
    assert lib.mg_create(2, 9, None, None, None, ctypes.byref(o), buf, 1 << 20, ctypes.byref(ctx)) == C.MG_EINVAL
    o.coarsest_n = 17  # above n
    assert lib.mg_create(2, 9, None, None, None, ctypes.byref(o), buf, 1 << 20, ctypes.byref(ctx)) == C.MG_EINVAL
    assert b"coarsest_n" in lib.mg_last_error()
    o.coarsest_n = 33  # 2^m+1, but no dense solve of that size
    assert lib.mg_workspace_bytes(2, 65, 0, ctypes.byref(o)) == 0
    lib.mg_default_options(ctypes.byref(o))
    assert lib.mg_create(2, 9, None, None, None, ctypes.byref(o), buf, 16, ctypes.byref(ctx)) == C.MG_ENOMEM
    assert lib.mg_create(2, 9, None, None, None, ctypes.byref(o), None, 1 << 20, ctypes.byref(ctx)) == C.MG_EINVAL
    assert lib.mg_destroy(None) == C.MG_OK
    assert lib.mg_num_levels(None) == -1


def test_missing_library_fails_loudly(tmp_path):
    from paper_1406_5369_gb300 import _capi
    saved = _capi._lib
    _capi._lib = None
    try:
        with pytest.raises(ImportError):
            _capi.load(str(tmp_path / "nope.so"))
    finally:
        _capi._lib = saved


def test_product_path_does_not_reach_the_oracle():
    pkg = os.path.join(ROOT, "paper_1406_5369_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, flags=re.M), fn
                for name in ("mg_oracle", "cc_oracle", "cd_oracle", "liboracle"):
                    assert name not in txt, (fn, name)


@pytest.mark.parametrize("dim", [2, 3])
def test_dense_coarsest_grid_adds_its_inverse_to_the_workspace(lib, dim):
    # coarsest_n 5 or 9: the hierarchy stops at that size and the arena holds
    # the FP64 inverse of the coarsest operator, N x N for N = (nc-2)^dim
    from paper_1406_5369_gb300 import _capi as C
    o = C.mg_options()
    lib.mg_default_options(ctypes.byref(o))
    n = 33 if dim == 3 else 65

    def a256(b):  # every arena buffer starts 256-byte aligned
        return -(-b // 256) * 256

    def fields(m):  # u[2], f, r of an m^dim FP64 level, 128-byte rows
        pitch = -(-m // 16) * 16
        return 4 * a256(pitch * m ** (dim - 1) * 8)

    base = lib.mg_workspace_bytes(dim, n, 0, ctypes.byref(o))
    for nc, dropped in [(5, [3]), (9, [5, 3])]:
        o.coarsest_n = nc
        got = lib.mg_workspace_bytes(dim, n, 0, ctypes.byref(o))
        N = (nc - 2) ** dim
        want = base - sum(fields(m) for m in dropped) + a256(N * N * 8)
        assert got == want, (nc, got, want)


def test_cell_grid_params_are_validated_without_a_device(lib):
    from paper_1406_5369_gb300 import _capi as C
    p = C.mg_cc_params()
    lib.mg_cc_default_params(ctypes.byref(p))
    assert (p.dim, p.n, p.sigma, p.bc, p.coarsest_n) == (2, 2, 1.0, C.MG_CC_NEUMANN, 1)
    p.n = 64
    good = lib.mg_cc_workspace_bytes(ctypes.byref(p))
    # levels 64..1: four FP64 fields each (rows padded to 16 doubles), the
    # 1x1 coarsest inverse, 4096 norm partials and the norm slot, 256-byte aligned
    a256 = lambda b: -(-b // 256) * 256
    want = sum(4 * a256(-(-m // 16) * 16 * m * 8) for m in (64, 32, 16, 8, 4, 2, 1)) + a256(8) + a256(4096 * 8) + 8
    assert good == a256(want)
    for field, bad in [("n", 48), ("n", 32768), ("dim", 4), ("sigma", -1.0), ("omega", 2.0), ("coarsest_n", 3),
                       ("coarsest_n", 128), ("bc", 5), ("nu1", 9)]:
        q = C.mg_cc_params()
        ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(p))
        setattr(q, field, bad)
        assert lib.mg_cc_workspace_bytes(ctypes.byref(q)) == 0, (field, bad)
    q = C.mg_cc_params()
    ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(p))
    q.sigma = 0.0  # singular with Neumann faces, fine with Dirichlet ones
    assert lib.mg_cc_workspace_bytes(ctypes.byref(q)) == 0
    assert b"Neumann" in lib.mg_last_error()
    q.bc = C.MG_CC_DIRICHLET
    assert lib.mg_cc_workspace_bytes(ctypes.byref(q)) == good
    ctx = ctypes.c_void_p()
    assert lib.mg_cc_create(ctypes.byref(p), ctypes.c_void_p(256), 16, ctypes.byref(ctx)) == C.MG_ENOMEM
    assert lib.mg_cc_num_levels(None) == -1


def test_complex_diffusion_params_are_validated_without_a_device(lib):
    from paper_1406_5369_gb300 import _capi as C
    p = C.mg_cd_params()
    lib.mg_cd_default_params(ctypes.byref(p))
    assert (p.n, p.nu1, p.nu2, p.smoother) == (2, 2, 2, C.MG_RBGS)
    p.n = 64
    good = lib.mg_cd_workspace_bytes(ctypes.byref(p))
    # levels 64..1: seven complex fields each (rows padded to 8 complex values),
    # 4096 norm partials and the norm slot, 256-byte aligned
    a256 = lambda b: -(-b // 256) * 256
    want = sum(7 * a256(-(-m // 8) * 8 * m * 16) for m in (64, 32, 16, 8, 4, 2, 1)) + a256(4096 * 8) + 8
    assert good == a256(want)
    for field, bad in [("n", 96), ("n", 16384), ("tau", 0.0), ("theta", 0.0), ("kappa", -1.0), ("omega", 0.0),
                       ("nu1", -1), ("maxit", -1), ("smoother", 7)]:
        q = C.mg_cd_params()
        ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(p))
        setattr(q, field, bad)
        assert lib.mg_cd_workspace_bytes(ctypes.byref(q)) == 0, (field, bad)
    ctx = ctypes.c_void_p()
    assert lib.mg_cd_create(ctypes.byref(p), ctypes.c_void_p(256), 16, ctypes.byref(ctx)) == C.MG_ENOMEM
    assert lib.mg_cd_num_levels(None) == -1


def test_solve_sequence_refuses_bad_arguments_without_a_device(lib):
    from paper_1406_5369_gb300 import _capi as C
    import ctypes
    st = lib.mg_solve_sequence(None, None, None, 1, None, None, 1e-8, None, None)
    assert st == C.MG_EINVAL
    assert b"contexts" in lib.mg_last_error()
