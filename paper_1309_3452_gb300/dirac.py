"""Python binding of libdirac (include/dirac.h): argument marshalling only.

Every step of the scheme runs in the CUDA library; this module converts
numpy arrays and workloads.Problem descriptions into the C ABI and raises on
any non-OK status.  Importing it loads libdirac.so and fails loudly when the
library has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libdirac.so not found at {LIB_PATH}; build it with "
                      "`python -m paper_1309_3452_gb300.build` (no CPU fallback exists)")

_lib = C.CDLL(LIB_PATH)

OK, ERR_INVALID, ERR_UNSTABLE, ERR_OOM, ERR_CUDA, ERR_DIVERGED, ERR_TIMEOUT, ERR_UNSUPPORTED = range(8)
FP64, FP32 = 0, 1
FLAG_ALLOW_UNSTABLE = 0x1
FLAG_REFERENCE_KERNELS = 0x2
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "UNSTABLE", 3: "OOM", 4: "CUDA", 5: "DIVERGED",
                6: "TIMEOUT", 7: "UNSUPPORTED"}


class DiracError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Fields(C.Structure):
    _fields_ = [
        ("V0", C.c_double), ("step_axis", C.c_int), ("step_x0", C.c_double), ("step_V", C.c_double),
        ("sc_Z", C.c_double), ("sc_a", C.c_double), ("sc_center", C.c_double * 3),
        ("V_static", C.POINTER(C.c_double)), ("Vmod_amp", C.c_double), ("Vmod_omega", C.c_double),
        ("q", C.c_double), ("A_const", C.c_double * 3), ("Apw_amp", C.c_double),
        ("Apw_k", C.c_double * 3), ("Apw_omega", C.c_double), ("Apw_phase", C.c_double),
        ("Apw_pol", C.c_int), ("V0_imag", C.c_double), ("abs_W", C.c_double), ("abs_width", C.c_double),
        ("abs_axes", C.c_int), ("A_links", C.POINTER(C.c_double)), ("Alink_amp", C.c_double),
        ("Alink_omega", C.c_double),
    ]


class Plan(C.Structure):
    _fields_ = [("chunk", C.c_int), ("two_step", C.c_int), ("chunk2", C.c_int), ("us_per_step", C.c_double)]

    def as_dict(self):
        return {"chunk": self.chunk, "two_step": self.two_step, "chunk2": self.chunk2,
                "us_per_step": self.us_per_step}


class CheckReport(C.Structure):
    _fields_ = [("E", C.c_double), ("naive", C.c_double), ("E_ref", C.c_double), ("naive_ref", C.c_double),
                ("drift", C.c_double), ("lower", C.c_double), ("upper", C.c_double), ("failed", C.c_uint)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


CHECK_NONFINITE, CHECK_BOUND, CHECK_DRIFT = 0x1, 0x2, 0x4

_vp = C.c_void_p
_dp = C.POINTER(C.c_double)
_lib.dirac_create.argtypes = [C.POINTER(_vp), C.c_int, C.POINTER(C.c_int), _dp, C.c_double,
                              C.c_double, C.POINTER(Fields), C.c_int, C.c_uint, _vp]
_lib.dirac_set_spinor.argtypes = [_vp, _dp]
_lib.dirac_get_spinor.argtypes = [_vp, _dp]
_lib.dirac_set_spinor_device.argtypes = [_vp, _vp]
_lib.dirac_get_spinor_device.argtypes = [_vp, _vp]
_lib.dirac_step.argtypes = [_vp, C.c_long]
_lib.dirac_batch_step.argtypes = [C.POINTER(_vp), C.c_int, C.c_long]
_lib.dirac_norm.argtypes = [_vp, _dp, _dp]
_lib.dirac_partial_density.argtypes = [_vp, C.c_int, C.c_double, _dp]
_lib.dirac_get_time.argtypes = [_vp, _dp]
_lib.dirac_set_time.argtypes = [_vp, C.c_double]
_lib.dirac_state_bytes.argtypes = [C.c_int, C.POINTER(C.c_int), C.c_int]
_lib.dirac_state_bytes.restype = C.c_size_t
_lib.dirac_last_error.argtypes = [_vp]
_lib.dirac_last_error.restype = C.c_char_p
_lib.dirac_destroy.argtypes = [_vp]
_lib.dirac_fields_default.argtypes = [C.POINTER(Fields)]
_lib.dirac_version.restype = C.c_int
# the structures above mirror include/dirac.h of this ABI version
ABI_VERSION = 2
if _lib.dirac_version() != ABI_VERSION:
    raise ImportError(f"{LIB_PATH} has ABI version {_lib.dirac_version()}, the binding expects "
                      f"{ABI_VERSION}; rebuild it with `python -m paper_1309_3452_gb300.build`")
_lib.dirac_get_plan.argtypes = [_vp, C.POINTER(Plan)]
_lib.dirac_set_plan.argtypes = [_vp, C.POINTER(Plan)]
_lib.dirac_autotune.argtypes = [_vp, C.POINTER(Plan)]
_lib.dirac_check.argtypes = [_vp, C.c_double, C.POINTER(CheckReport)]
_lib.dirac_functional_bounds.argtypes = [C.c_int, _dp, C.c_double, C.c_int, _dp, _dp]
_lib.dirac_functional_bounds.restype = None
_lib.dirac_algorithmic_bytes.argtypes = [_vp]
_lib.dirac_algorithmic_bytes.restype = C.c_double
_lib.dirac_kernel_launches.argtypes = [_vp]
_lib.dirac_kernel_launches.restype = C.c_longlong

for _name in ("dirac_create", "dirac_set_spinor", "dirac_get_spinor", "dirac_set_spinor_device",
              "dirac_get_spinor_device", "dirac_step", "dirac_batch_step", "dirac_norm",
              "dirac_partial_density", "dirac_get_time", "dirac_set_time", "dirac_get_plan",
              "dirac_set_plan", "dirac_autotune", "dirac_check"):
    getattr(_lib, _name).restype = C.c_int


_lib.dirac_slab_partition.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
_lib.dirac_slab_partition.restype = None
_lib.dirac_slabs_create.argtypes = [C.POINTER(_vp), C.c_int, C.c_int, C.POINTER(C.c_int), _dp, C.c_double,
                                    C.c_double, C.POINTER(Fields), C.c_int, C.c_uint, _vp]
_lib.dirac_slabs_set_spinor.argtypes = [_vp, _dp]
_lib.dirac_slabs_get_spinor.argtypes = [_vp, _dp]
_lib.dirac_slabs_step.argtypes = [_vp, C.c_long]
_lib.dirac_slabs_norm.argtypes = [_vp, _dp, _dp]
_lib.dirac_slabs_info.argtypes = [_vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
_lib.dirac_slabs_get_time.argtypes = [_vp, _dp]
_lib.dirac_slabs_kernel_launches.argtypes = [_vp]
_lib.dirac_slabs_kernel_launches.restype = C.c_longlong
_lib.dirac_slabs_last_error.argtypes = [_vp]
_lib.dirac_slabs_last_error.restype = C.c_char_p
_lib.dirac_slabs_destroy.argtypes = [_vp]
for _name in ("dirac_slabs_create", "dirac_slabs_set_spinor", "dirac_slabs_get_spinor", "dirac_slabs_step",
              "dirac_slabs_norm", "dirac_slabs_info", "dirac_slabs_get_time"):
    getattr(_lib, _name).restype = C.c_int


_lib.dirac_fp64_fma_rate.argtypes = [_dp]
_lib.dirac_fp64_fma_rate.restype = C.c_int


def lib():
    return _lib


def fp64_fma_rate():
    """Measured FP64 FMA rate of the current device, TFLOP/s (dirac_fp64_fma_rate)."""
    r = C.c_double()
    rc = _lib.dirac_fp64_fma_rate(C.byref(r))
    if rc != OK:
        raise DiracError(rc, _lib.dirac_last_error(None).decode())
    return r.value


def slab_partition(Nz, nslabs):
    """[(z0, nz)] of the slabs dirac_slabs_create uses (host only)."""
    out = []
    for k in range(nslabs):
        z0, nz = C.c_int(), C.c_int()
        _lib.dirac_slab_partition(int(Nz), int(nslabs), k, C.byref(z0), C.byref(nz))
        out.append((z0.value, nz.value))
    return out


def _fields_struct(f):
    s = Fields()
    _lib.dirac_fields_default(C.byref(s))
    if f is None:
        return s, {}
    s.V0 = f.V0
    s.step_axis, s.step_x0, s.step_V = int(f.step_axis), float(f.step_x0), float(f.step_V)
    s.sc_Z, s.sc_a = float(f.sc_Z), float(f.sc_a)
    for a in range(3):
        s.sc_center[a] = float(f.sc_center[a]) if a < len(f.sc_center) else 0.0
        s.A_const[a] = float(f.A_const[a]) if a < len(f.A_const) else 0.0
        s.Apw_k[a] = float(f.Apw_k[a]) if a < len(f.Apw_k) else 0.0
    keep = {}
    if f.V_static is not None:
        keep["V_static"] = np.ascontiguousarray(f.V_static, dtype=np.float64)
        s.V_static = keep["V_static"].ctypes.data_as(_dp)
    if getattr(f, "A_links", None) is not None:
        keep["A_links"] = np.ascontiguousarray(f.A_links, dtype=np.float64)
        s.A_links = keep["A_links"].ctypes.data_as(_dp)
    s.Alink_amp = float(getattr(f, "Alink_amp", 0.0))
    s.Alink_omega = float(getattr(f, "Alink_omega", 0.0))
    s.Vmod_amp, s.Vmod_omega = float(f.Vmod_amp), float(f.Vmod_omega)
    s.q = float(f.q)
    s.Apw_amp, s.Apw_omega, s.Apw_phase = float(f.Apw_amp), float(f.Apw_omega), float(f.Apw_phase)
    s.Apw_pol = int(f.Apw_pol)
    s.V0_imag = float(f.V0_imag)
    s.abs_W, s.abs_width, s.abs_axes = float(f.abs_W), float(f.abs_width), int(f.abs_axes)
    return s, keep


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def batch_step(sims, nsteps):
    """Advance several Sim objects together (dirac_batch_step)."""
    if not sims:
        return
    arr = (_vp * len(sims))(*[s._h for s in sims])
    rc = _lib.dirac_batch_step(arr, len(sims), int(nsteps))
    if rc != OK:
        raise DiracError(rc, _lib.dirac_last_error(None).decode())


def functional_bounds(dims, dx, dt, general_A=False):
    """(lo, hi) with lo sum|psi|^2 <= E <= hi sum|psi|^2 (dirac_functional_bounds)."""
    d = (C.c_double * 3)(*[float(v) for v in (list(dx) + [1.0, 1.0, 1.0])[:3]])
    lo, hi = C.c_double(), C.c_double()
    _lib.dirac_functional_bounds(int(dims), d, float(dt), int(bool(general_A)), C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def state_bytes(dims, N, precision):
    n = (C.c_int * 3)(*[int(v) for v in (list(N) + [1, 1, 1])[:3]])
    return int(_lib.dirac_state_bytes(int(dims), n, int(precision)))


class Sim:
    """One simulation owned by libdirac.  `prob` is a workloads.Problem."""

    def __init__(self, prob, precision=FP64, flags=0, stream=None):
        self.prob = prob
        self.precision = precision
        n = (C.c_int * 3)(*[int(v) for v in (list(prob.N) + [1, 1, 1])[:3]])
        dx = (C.c_double * 3)(*[float(v) for v in (list(prob.dx) + [1.0, 1.0, 1.0])[:3]])
        fs, keep = _fields_struct(prob.fields)
        if "V_static" in keep and keep["V_static"].size != int(np.prod(prob.shape)):
            raise ValueError("V_static must have one value per site (canonical layout)")
        if "A_links" in keep and keep["A_links"].size != int(prob.dims) * int(np.prod(prob.shape)):
            raise ValueError("A_links must have dims values per site (axis-major, canonical layout)")
        self._h = _vp()
        st = stream if stream is not None else _current_stream()
        rc = _lib.dirac_create(C.byref(self._h), int(prob.dims), n, dx, float(prob.dt), float(prob.m),
                               C.byref(fs), int(precision), int(flags), st)
        if rc != OK:
            raise DiracError(rc, _lib.dirac_last_error(None).decode())
        del keep

    def _check(self, rc):
        if rc != OK:
            raise DiracError(rc, _lib.dirac_last_error(self._h).decode())

    def set_spinor(self, psi):
        a = np.ascontiguousarray(psi, dtype=np.complex128)
        if a.size != int(np.prod(self.prob.shape)):
            raise ValueError("state has the wrong number of values")
        self._check(_lib.dirac_set_spinor(self._h, a.ctypes.data_as(_dp)))

    def set_spinor_ptr(self, host_ptr: int):
        """Canonical complex128 state at a raw host address (e.g. pinned memory)."""
        self._check(_lib.dirac_set_spinor(self._h, C.cast(C.c_void_p(host_ptr), _dp)))

    def set_spinor_device(self, dev_ptr: int):
        """Canonical complex128 state in device memory (e.g. a torch tensor's data_ptr())."""
        self._check(_lib.dirac_set_spinor_device(self._h, _vp(dev_ptr)))

    def get_spinor_device(self, dev_ptr: int):
        self._check(_lib.dirac_get_spinor_device(self._h, _vp(dev_ptr)))

    def get_spinor(self):
        out = np.empty(self.prob.shape, np.complex128)
        self._check(_lib.dirac_get_spinor(self._h, out.ctypes.data_as(_dp)))
        return out

    def get_spinor_ptr(self, host_ptr: int):
        self._check(_lib.dirac_get_spinor(self._h, C.cast(C.c_void_p(host_ptr), _dp)))

    def step(self, n):
        self._check(_lib.dirac_step(self._h, int(n)))

    def norm(self):
        E, naive = C.c_double(), C.c_double()
        self._check(_lib.dirac_norm(self._h, C.byref(E), C.byref(naive)))
        return E.value, naive.value

    def partial_density(self, axis, x0):
        out = C.c_double()
        self._check(_lib.dirac_partial_density(self._h, int(axis), float(x0), C.byref(out)))
        return out.value

    @property
    def launches(self):
        return int(_lib.dirac_kernel_launches(self._h))

    def check(self, tol=1e-6):
        """dirac_check: (ok, report).  ok is False when a check failed
        (DIRAC_ERR_DIVERGED); any other failure raises."""
        r = CheckReport()
        rc = _lib.dirac_check(self._h, float(tol), C.byref(r))
        if rc not in (OK, ERR_DIVERGED):
            self._check(rc)
        return rc == OK, r.as_dict()

    @property
    def algorithmic_bytes(self):
        """HBM bytes per site update on this simulation's path (dirac_algorithmic_bytes)."""
        return float(_lib.dirac_algorithmic_bytes(self._h))

    @property
    def plan(self):
        p = Plan()
        self._check(_lib.dirac_get_plan(self._h, C.byref(p)))
        return p.as_dict()

    def set_plan(self, chunk=0, two_step=0, chunk2=0):
        p = Plan(int(chunk), int(two_step), int(chunk2), 0.0)
        self._check(_lib.dirac_set_plan(self._h, C.byref(p)))

    def autotune(self):
        """Time the candidate launch plans on the current state and keep the
        fastest (dirac_autotune); returns the plan."""
        p = Plan()
        self._check(_lib.dirac_autotune(self._h, C.byref(p)))
        return p.as_dict()

    @property
    def time(self):
        t = C.c_double()
        self._check(_lib.dirac_get_time(self._h, C.byref(t)))
        return t.value

    @time.setter
    def time(self, t):
        self._check(_lib.dirac_set_time(self._h, float(t)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.dirac_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Slabs:
    """A (3+1)D grid split along z into slabs stepped as sub-domains with halo
    exchange (dirac_slabs_*); the same calls as Sim for the whole grid."""

    def __init__(self, prob, nslabs, precision=FP32, flags=0, stream=None):
        self.prob = prob
        n = (C.c_int * 3)(*[int(v) for v in (list(prob.N) + [1, 1, 1])[:3]])
        dx = (C.c_double * 3)(*[float(v) for v in (list(prob.dx) + [1.0, 1.0, 1.0])[:3]])
        fs, keep = _fields_struct(prob.fields)
        self._h = _vp()
        st = stream if stream is not None else _current_stream()
        rc = _lib.dirac_slabs_create(C.byref(self._h), int(nslabs), int(prob.dims), n, dx, float(prob.dt),
                                     float(prob.m), C.byref(fs), int(precision), int(flags), st)
        if rc != OK:
            raise DiracError(rc, _lib.dirac_slabs_last_error(None).decode())
        self.nslabs = int(nslabs)
        del keep

    def _check(self, rc):
        if rc != OK:
            raise DiracError(rc, _lib.dirac_slabs_last_error(self._h).decode())

    def set_spinor(self, psi):
        a = np.ascontiguousarray(psi, dtype=np.complex128)
        if a.size != int(np.prod(self.prob.shape)):
            raise ValueError("state has the wrong number of values")
        self._check(_lib.dirac_slabs_set_spinor(self._h, a.ctypes.data_as(_dp)))

    def get_spinor(self):
        out = np.empty(self.prob.shape, np.complex128)
        self._check(_lib.dirac_slabs_get_spinor(self._h, out.ctypes.data_as(_dp)))
        return out

    def step(self, n):
        self._check(_lib.dirac_slabs_step(self._h, int(n)))

    def norm(self):
        E, naive = C.c_double(), C.c_double()
        self._check(_lib.dirac_slabs_norm(self._h, C.byref(E), C.byref(naive)))
        return E.value, naive.value

    def info(self, k):
        z0, nz = C.c_int(), C.c_int()
        self._check(_lib.dirac_slabs_info(self._h, int(k), C.byref(z0), C.byref(nz)))
        return z0.value, nz.value

    @property
    def time(self):
        t = C.c_double()
        self._check(_lib.dirac_slabs_get_time(self._h, C.byref(t)))
        return t.value

    @property
    def launches(self):
        return int(_lib.dirac_slabs_kernel_launches(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.dirac_slabs_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
