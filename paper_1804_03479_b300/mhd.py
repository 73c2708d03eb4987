"""Thin ctypes binding of libmhd.so (include/mhd.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  If the library cannot be loaded this module raises; there is
no fallback path.  Arrays may be numpy arrays (host) or torch tensors (host
or CUDA); the state layout is that of include/mhd.h: U (5, nz, ny, nx) and
B (3, nz, ny, nx), float64 for fp64/mixed and float32 for fp32.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmhd.so")

MHD_OK, MHD_EINVAL, MHD_ENOMEM, MHD_ECUDA, MHD_ENEGATIVE, MHD_ETIMEOUT, MHD_EUNSUPPORTED = range(7)
STATUS = {0: "MHD_OK", 1: "MHD_EINVAL", 2: "MHD_ENOMEM", 3: "MHD_ECUDA", 4: "MHD_ENEGATIVE",
          5: "MHD_ETIMEOUT", 6: "MHD_EUNSUPPORTED"}
INTEGRATORS = {"vl": 0, "ctu": 1}
RECONS = {"plm": 0, "ppm": 1, "plm_prim": 2}
SOLVERS = {"roe": 0, "hlld": 1, "hlle": 2}
PRECISIONS = {"fp64": 0, "fp32": 1, "mixed": 2}

EXPORTS = ["mhd_init", "mhd_set_state", "mhd_get_state", "mhd_cfl_dt", "mhd_step", "mhd_advance",
           "mhd_last_dt", "mhd_divB", "mhd_sums", "mhd_sync", "mhd_bad_cell", "mhd_clear_error",
           "mhd_last_error", "mhd_device_bytes", "mhd_launches_per_step", "mhd_free",
           "mhd_profile_begin", "mhd_profile_end", "mhd_step_noalloc"]
GROUPS = ["prim_cfl", "predictor_sweeps", "emf1", "half_update", "corrector_sweeps", "emf2", "full_update"]


class MHDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("dx", ctypes.c_double)]


class Scheme(ctypes.Structure):
    _fields_ = [("integrator", ctypes.c_int), ("recon", ctypes.c_int), ("riemann", ctypes.c_int),
                ("precision", ctypes.c_int), ("cfl", ctypes.c_double)]


_lib = None


def lib():
    """Load libmhd.so (raises OSError if it is missing: build it first)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError(f"{LIB_PATH} not found: run `python -m paper_1804_03479_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    L.mhd_init.argtypes = [ctypes.POINTER(Grid), ctypes.c_double, ctypes.POINTER(Scheme), vp, ctypes.POINTER(vp)]
    L.mhd_set_state.argtypes = [vp, vp, vp, ip]
    L.mhd_get_state.argtypes = [vp, vp, vp, ip]
    L.mhd_cfl_dt.argtypes = [vp, dp]
    L.mhd_step.argtypes = [vp, ctypes.c_double]
    L.mhd_advance.argtypes = [vp, ip, ip]
    L.mhd_last_dt.argtypes = [vp, dp]
    L.mhd_divB.argtypes = [vp, dp, dp]
    L.mhd_sums.argtypes = [vp, dp]
    L.mhd_sync.argtypes = [vp]
    L.mhd_bad_cell.argtypes = [vp]
    L.mhd_bad_cell.restype = ctypes.c_longlong
    L.mhd_clear_error.argtypes = [vp]
    L.mhd_clear_error.restype = None
    L.mhd_last_error.argtypes = [vp]
    L.mhd_last_error.restype = ctypes.c_char_p
    L.mhd_device_bytes.argtypes = [vp]
    L.mhd_device_bytes.restype = ctypes.c_longlong
    L.mhd_launches_per_step.argtypes = [vp]
    L.mhd_free.argtypes = [vp]
    L.mhd_free.restype = None
    L.mhd_step_noalloc.argtypes = [ctypes.POINTER(Grid), ctypes.c_double, ctypes.POINTER(Scheme), ctypes.c_double,
                                   vp, vp, vp]
    L.mhd_step_noalloc.restype = ctypes.c_int
    L.mhd_profile_begin.argtypes = [vp, ip]
    L.mhd_profile_end.argtypes = [vp, dp, ip, ctypes.POINTER(ctypes.c_int)]
    for name in ["mhd_init", "mhd_set_state", "mhd_get_state", "mhd_cfl_dt", "mhd_step", "mhd_advance",
                 "mhd_last_dt", "mhd_divB", "mhd_sums", "mhd_sync", "mhd_launches_per_step",
                 "mhd_profile_begin", "mhd_profile_end", "mhd_step_noalloc"]:
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _ptr(a):
    """(address, on_device) of a numpy array or torch tensor (contiguous)."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data, 0
    assert a.is_contiguous()
    return a.data_ptr(), int(a.is_cuda)


NOALLOC_MAX_CELLS = 32768


def step_noalloc(U, B, dx, dt, gamma=5.0 / 3.0, recon="plm", riemann="roe", stream=None):
    """One FP64 VL step of a caller-owned device state (torch CUDA float64
    tensors U (5, nz, ny, nx) and B (3, nz, ny, nx)), in place, through
    mhd_step_noalloc: no device memory is allocated (the scratch is a fixed
    array inside the library, at most NOALLOC_MAX_CELLS cells).  Calls that
    overlap on the GPU share that array and race: serialise them."""
    nz, ny, nx = U.shape[1:]
    g = Grid(nx, ny, nz, dx)
    s = Scheme(INTEGRATORS["vl"], RECONS[recon], SOLVERS[riemann], PRECISIONS["fp64"], 0.3)
    pu, du = _ptr(U)
    pb, db = _ptr(B)
    if not (du and db):
        raise MHDError(MHD_EINVAL, "step_noalloc takes device arrays")
    st = lib().mhd_step_noalloc(ctypes.byref(g), gamma, ctypes.byref(s), dt, ctypes.c_void_p(pu),
                                ctypes.c_void_p(pb), ctypes.c_void_p(stream or 0))
    if st != MHD_OK:
        raise MHDError(st, lib().mhd_last_error(None).decode())


class Solver:
    """One periodic box advanced by the library (one mhd_ctx)."""

    def __init__(self, shape, dx, gamma=5.0 / 3.0, integrator="vl", recon="plm", riemann="roe",
                 precision="fp64", cfl=0.3, stream=None):
        self.nz, self.ny, self.nx = shape if len(shape) == 3 else shape[-3:]
        self.precision = precision
        self.dtype = np.float32 if precision == "fp32" else np.float64
        g = Grid(self.nx, self.ny, self.nz, dx)
        s = Scheme(INTEGRATORS[integrator], RECONS[recon], SOLVERS[riemann], PRECISIONS[precision], cfl)
        h = ctypes.c_void_p()
        st = lib().mhd_init(ctypes.byref(g), gamma, ctypes.byref(s), ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if st != MHD_OK:
            raise MHDError(st, lib().mhd_last_error(None).decode())
        self.h = h
        self.n = self.nx * self.ny * self.nz

    def _check(self, st):
        if st != MHD_OK:
            raise MHDError(st, lib().mhd_last_error(self.h).decode())

    def set_state(self, U, B):
        pu, du = _ptr(U)
        pb, db = _ptr(B)
        assert du == db
        self._check(lib().mhd_set_state(self.h, ctypes.c_void_p(pu), ctypes.c_void_p(pb), du))

    def get_state(self, U=None, B=None):
        if U is None:
            U = np.empty((5, self.nz, self.ny, self.nx), self.dtype)
            B = np.empty((3, self.nz, self.ny, self.nx), self.dtype)
        pu, du = _ptr(U)
        pb, db = _ptr(B)
        self._check(lib().mhd_get_state(self.h, ctypes.c_void_p(pu), ctypes.c_void_p(pb), du))
        return U, B

    def cfl_dt(self):
        dt = ctypes.c_double()
        self._check(lib().mhd_cfl_dt(self.h, ctypes.byref(dt)))
        return dt.value

    def step(self, dt):
        self._check(lib().mhd_step(self.h, dt))

    def advance(self, nsteps, use_graph=False):
        self._check(lib().mhd_advance(self.h, nsteps, int(use_graph)))

    def last_dt(self):
        dt = ctypes.c_double()
        self._check(lib().mhd_last_dt(self.h, ctypes.byref(dt)))
        return dt.value

    def divB(self):
        m, r = ctypes.c_double(), ctypes.c_double()
        self._check(lib().mhd_divB(self.h, ctypes.byref(m), ctypes.byref(r)))
        return m.value, r.value

    def sums(self):
        out = (ctypes.c_double * 8)()
        self._check(lib().mhd_sums(self.h, out))
        return np.array(out[:])

    def sync(self):
        self._check(lib().mhd_sync(self.h))

    def bad_cell(self):
        return lib().mhd_bad_cell(self.h)

    def clear_error(self):
        lib().mhd_clear_error(self.h)

    def device_bytes(self):
        return lib().mhd_device_bytes(self.h)

    def launches_per_step(self):
        return lib().mhd_launches_per_step(self.h)

    def profile_begin(self, max_steps):
        self._check(lib().mhd_profile_begin(self.h, max_steps))

    def profile_end(self):
        """summed ms per kernel group (GROUPS) and the number of steps recorded"""
        ms = (ctypes.c_double * 7)()
        steps = ctypes.c_int()
        self._check(lib().mhd_profile_end(self.h, ms, 7, ctypes.byref(steps)))
        return dict(zip(GROUPS, ms[:])), steps.value

    def free(self):
        if getattr(self, "h", None):
            lib().mhd_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
