"""The C-ABI library builds, loads without a GPU and exports every function
include/dirac.h declares; host-only argument validation works on the CPU."""
import ctypes as C
import os
import re

import pytest

from paper_1309_3452_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(dirac_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    return C.CDLL(B.build())


def test_header_declares_the_api():
    names = declared_functions()
    for want in ("dirac_create", "dirac_set_spinor", "dirac_get_spinor", "dirac_step", "dirac_norm",
                 "dirac_partial_density", "dirac_destroy", "dirac_last_error"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_validation(lib):
    from paper_1309_3452_gb300 import dirac as D

    assert D.lib().dirac_version() == D.ABI_VERSION == 2
    f = D.Fields()
    D.lib().dirac_fields_default(C.byref(f))
    assert f.q == 1.0 and f.step_axis == -1 and f.sc_a == 1.0 and f.V0 == 0.0
    h = C.c_void_p()
    N = (C.c_int * 3)(8, 8, 8)
    dx = (C.c_double * 3)(1.0, 1.0, 1.0)
    L = D.lib()
    # rejected before any CUDA call
    assert L.dirac_create(C.byref(h), 4, N, dx, 0.5, 0.0, None, 0, 0, None) == D.ERR_INVALID
    assert L.dirac_create(C.byref(h), 3, N, dx, 0.6, 0.0, None, 0, 0, None) == D.ERR_UNSTABLE
    assert b"stability" in L.dirac_last_error(None)
    bad = (C.c_int * 3)(1, 8, 8)
    assert L.dirac_create(C.byref(h), 3, bad, dx, 0.5, 0.0, None, 0, 0, None) == D.ERR_INVALID
    assert L.dirac_create(C.byref(h), 2, N, dx, -0.1, 0.0, None, 0, 0, None) == D.ERR_INVALID
    # the stability bound sum_a (dt/dx_a)^2 <= 1 with per-axis spacings
    adx = (C.c_double * 3)(1.0, 1.3, 0.8)
    dt_max = 1.0 / (1.0 + 1.0 / 1.3 ** 2 + 1.0 / 0.8 ** 2) ** 0.5
    assert L.dirac_create(C.byref(h), 3, N, adx, 1.01 * dt_max, 0.0, None, 0, 0, None) == D.ERR_UNSTABLE
    rc = L.dirac_create(C.byref(h), 3, N, adx, 0.99 * dt_max, 0.0, None, 0, 0, None)
    assert rc != D.ERR_UNSTABLE  # accepted (without a device creation then fails later, with ERR_CUDA)
    if rc == D.OK:
        L.dirac_destroy(h)
        h = C.c_void_p()
    # absorbing layers: a width and a non-empty mask of the grid's axes
    for width, axes, dims in ((0.0, 1, 3), (2.0, 0, 3), (2.0, 8, 3), (2.0, 4, 2)):
        g = D.Fields()
        L.dirac_fields_default(C.byref(g))
        g.abs_W, g.abs_width, g.abs_axes = 0.5, width, axes
        assert L.dirac_create(C.byref(h), dims, N, dx, 0.5, 0.0, C.byref(g), 0, 0, None) == D.ERR_INVALID
    assert b"abs_axes" in L.dirac_last_error(None)
    # link integrals need a finite modulation and charge
    links = (C.c_double * (3 * 8 * 512))()
    g = D.Fields()
    L.dirac_fields_default(C.byref(g))
    g.A_links = C.cast(links, C.POINTER(C.c_double))
    g.Alink_amp = float("nan")
    assert L.dirac_create(C.byref(h), 3, N, dx, 0.5, 0.0, C.byref(g), 0, 0, None) == D.ERR_INVALID
    assert b"Alink_amp" in L.dirac_last_error(None)
    # the allocation-free norm cannot take link integrals (rejected before any device work)
    g.Alink_amp = 0.0
    L.dirac_norm_noalloc.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_double,
                                     C.c_double, C.c_void_p, C.c_int, C.POINTER(C.c_void_p),
                                     C.c_void_p, C.c_void_p]
    dummy = (C.c_void_p * 8)(*([16] * 8))  # never dereferenced
    assert L.dirac_norm_noalloc(3, N, dx, 0.5, 0.0, C.byref(g), D.FP32, dummy, 16, None) == D.ERR_UNSUPPORTED
    # a non-finite Klein-step position or height is refused before any device work (a NaN
    # threshold would otherwise never be found)
    for name, val in (("step_x0", float("nan")), ("step_x0", float("inf")), ("step_x0", -float("inf")),
                      ("step_V", float("nan")), ("sc_center", float("inf"))):
        g = D.Fields()
        L.dirac_fields_default(C.byref(g))
        g.step_axis, g.step_x0, g.step_V = 0, 4.25, 0.5
        if name == "sc_center":
            g.sc_Z = 1.0
            g.sc_center[1] = val
        else:
            setattr(g, name, val)
        assert L.dirac_create(C.byref(h), 3, N, dx, 0.5, 0.0, C.byref(g), 0, 0, None) == D.ERR_INVALID
        assert name.encode() in L.dirac_last_error(None)
    # a huge but finite step position is accepted (no site lies beyond it)
    g = D.Fields()
    L.dirac_fields_default(C.byref(g))
    g.step_axis, g.step_x0, g.step_V = 0, 1e300, 0.5
    rc = L.dirac_create(C.byref(h), 3, N, dx, 0.5, 0.0, C.byref(g), 0, 0, None)
    assert rc in (D.OK, D.ERR_CUDA)
    if rc == D.OK:
        L.dirac_destroy(h)
        h = C.c_void_p()
    # the allocation-free norm checks the vector potential as dirac_create does
    for setup in ("pol", "nan_q", "inf_A", "nan_k"):
        g = D.Fields()
        L.dirac_fields_default(C.byref(g))
        if setup == "pol":
            g.Apw_amp, g.Apw_pol = 0.3, 3
        elif setup == "nan_q":
            g.q = float("nan")
        elif setup == "inf_A":
            g.A_const[2] = float("inf")
        else:
            g.Apw_amp, g.Apw_k[0] = 0.3, float("nan")
        assert L.dirac_norm_noalloc(3, N, dx, 0.5, 0.0, C.byref(g), D.FP32, dummy, 16, None) == D.ERR_INVALID
    g = D.Fields()
    L.dirac_fields_default(C.byref(g))
    g.Apw_amp, g.Apw_pol = 0.3, 2
    assert L.dirac_norm_noalloc(2, N, dx, 0.5, 0.0, C.byref(g), D.FP32, dummy, 16, None) == D.ERR_INVALID
    # grids beyond the 32-bit row indexing of the kernels are refused before any device work
    big = (C.c_int * 3)(65536, 32768, 1)
    assert L.dirac_create(C.byref(h), 2, big, dx, 0.5, 0.0, None, 1, 0, None) == D.ERR_UNSUPPORTED
    assert b"2^31" in L.dirac_last_error(None)
    assert not h.value
    # device bytes: 8 planes x 8^3 cells x complex128
    assert D.state_bytes(3, (8, 8, 8), D.FP64) == 8 * 512 * 16
    assert D.state_bytes(2, (10, 10), D.FP32) == 2 * 4 * 128 * 8 + 128 * 16
