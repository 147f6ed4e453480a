"""ctypes wrapper of the FP64 CPU oracle (dirac_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and
by bench.py's CPU-baseline leg.  The library path never imports it.

The wrapper takes a workloads.Problem and a canonical complex128 state of
shape (P, Nz, Ny, Nx); it never touches the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dirac_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "libdirac_oracle.so")

# -ffp-contract=off: no fused multiply-add, every operation rounds as written.
# -fcx-limited-range: textbook complex multiply/divide (no NaN recovery calls).
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fcx-limited-range",
          "-fno-fast-math"]

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available).  Returns the path."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "dirac_oracle.h"))):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    base = ["gcc"] + CFLAGS + ["-o", tmp, SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, LIB)
    return LIB


class _Problem(C.Structure):
    _fields_ = [
        ("dims", C.c_int), ("N", C.c_int * 3), ("dx", C.c_double * 3), ("dt", C.c_double),
        ("m", C.c_double), ("V0", C.c_double), ("step_axis", C.c_int), ("step_x0", C.c_double),
        ("step_V", C.c_double), ("sc_Z", C.c_double), ("sc_a", C.c_double),
        ("sc_c", C.c_double * 3), ("V_site", C.POINTER(C.c_double)), ("Vmod_amp", C.c_double),
        ("Vmod_omega", C.c_double), ("q", C.c_double), ("A_const", C.c_double * 3),
        ("Apw_amp", C.c_double), ("Apw_k", C.c_double * 3), ("Apw_omega", C.c_double),
        ("Apw_phase", C.c_double), ("Apw_pol", C.c_int), ("origin", C.c_int * 3),
        ("V0_imag", C.c_double), ("abs_W", C.c_double), ("abs_width", C.c_double), ("abs_axes", C.c_int),
        ("A_links", C.POINTER(C.c_double)), ("Alink_amp", C.c_double), ("Alink_omega", C.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            _lib.oracle_step.argtypes = [C.POINTER(_Problem), dp, C.c_double, C.c_long]
            _lib.oracle_observables.argtypes = [C.POINTER(_Problem), dp, C.c_double, dp]
            _lib.oracle_partial_density.argtypes = [C.POINTER(_Problem), dp, C.c_int, C.c_double]
            _lib.oracle_partial_density.restype = C.c_double
            _lib.oracle_threads.restype = C.c_int
    return _lib


def _problem(prob, origin=(0, 0, 0)):
    f = prob.fields
    p = _Problem()
    p.dims = prob.dims
    for a in range(3):
        p.N[a] = int(prob.N[a]) if a < len(prob.N) else 1
        p.dx[a] = float(prob.dx[a]) if a < len(prob.dx) else 1.0
        p.sc_c[a] = float(f.sc_center[a]) if a < len(f.sc_center) else 0.0
        p.A_const[a] = float(f.A_const[a]) if a < len(f.A_const) else 0.0
        p.Apw_k[a] = float(f.Apw_k[a]) if a < len(f.Apw_k) else 0.0
        p.origin[a] = int(origin[a])
    p.dt, p.m, p.V0 = float(prob.dt), float(prob.m), float(f.V0)
    p.step_axis, p.step_x0, p.step_V = int(f.step_axis), float(f.step_x0), float(f.step_V)
    p.sc_Z, p.sc_a = float(f.sc_Z), float(f.sc_a)
    keep = None
    if f.V_static is not None:
        keep = np.ascontiguousarray(f.V_static, dtype=np.float64).reshape(prob.shape)
        p.V_site = keep.ctypes.data_as(C.POINTER(C.c_double))
    p.Vmod_amp, p.Vmod_omega = float(f.Vmod_amp), float(f.Vmod_omega)
    p.q = float(f.q)
    p.Apw_amp, p.Apw_omega, p.Apw_phase = float(f.Apw_amp), float(f.Apw_omega), float(f.Apw_phase)
    p.Apw_pol = int(f.Apw_pol)
    p.V0_imag = float(f.V0_imag)
    p.abs_W, p.abs_width, p.abs_axes = float(f.abs_W), float(f.abs_width), int(f.abs_axes)
    if p.abs_W != 0.0 and any(origin):
        raise ValueError("absorbing layers refer to the grid's own box: no window origin")
    if f.A_links is not None:
        links = np.ascontiguousarray(f.A_links, dtype=np.float64).reshape((prob.dims,) + tuple(prob.shape))
        p.A_links = links.ctypes.data_as(C.POINTER(C.c_double))
        keep = (keep, links)
    p.Alink_amp, p.Alink_omega = float(f.Alink_amp), float(f.Alink_omega)
    return p, keep


def _state(prob, psi):
    a = np.ascontiguousarray(psi, dtype=np.complex128).reshape(prob.shape).copy()
    return a


def step(prob, psi, nsteps: int, t0: float = 0.0, origin=(0, 0, 0)) -> np.ndarray:
    """Return the state after nsteps full steps starting at lower-sheet time t0."""
    p, keep = _problem(prob, origin)
    a = _state(prob, psi)
    lib().oracle_step(C.byref(p), a.ctypes.data_as(C.POINTER(C.c_double)), float(t0), int(nsteps))
    del keep
    return a


def observables(prob, psi, t: float = 0.0, origin=(0, 0, 0)) -> dict:
    """E (lower form), E_upper (the Lemma's upper form) and the naive norm."""
    p, keep = _problem(prob, origin)
    a = _state(prob, psi)
    out = (C.c_double * 3)()
    lib().oracle_observables(C.byref(p), a.ctypes.data_as(C.POINTER(C.c_double)), float(t), out)
    del keep
    return {"E": out[0], "E_upper": out[1], "naive": out[2]}


def partial_density(prob, psi, axis: int, x0: float, origin=(0, 0, 0)) -> float:
    p, keep = _problem(prob, origin)
    a = _state(prob, psi)
    r = lib().oracle_partial_density(C.byref(p), a.ctypes.data_as(C.POINTER(C.c_double)), int(axis),
                                     float(x0))
    del keep
    return r


def threads() -> int:
    return int(lib().oracle_threads())
