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
           "mhd_profile_begin", "mhd_profile_end", "mhd_step_noalloc", "mhd_init_batch", "mhd_nbox",
           "mhd_set_state_box", "mhd_get_state_box", "mhd_step_boxes", "mhd_set_sweep_config",
           "mhd_get_sweep_config", "mhd_autotune", "mhd_mlp_create", "mhd_mlp_free", "mhd_mlp_nparam",
           "mhd_mlp_set_weights", "mhd_mlp_get_weights", "mhd_mlp_grad", "mhd_mlp_train_step",
           "mhd_mlp_predict", "mhd_nblocks", "mhd_block_features", "mhd_block_error", "mhd_set_selector",
           "mhd_selector_stats", "mhd_floor_count", "mhd_energies", "mhd_helicity",
           "mhd_set_sweep_pencils", "mhd_get_sweep_pencils", "mhd_set_boundary", "mhd_get_boundary",
           "mhd_pressure_gradient", "mhd_set_dirichlet", "mhd_get_dirichlet", "mhd_set_emf_staging",
           "mhd_get_emf_staging", "mhd_inject_wait_flag", "mhd_fma_peak"]
GROUPS = ["prim_cfl", "predictor_x", "predictor_y", "predictor_z", "emf1", "half_update", "corrector_x",
          "corrector_y", "corrector_z", "emf2", "full_update"]


class MHDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("dx", ctypes.c_double)]


class Scheme(ctypes.Structure):
    _fields_ = [("integrator", ctypes.c_int), ("recon", ctypes.c_int), ("riemann", ctypes.c_int),
                ("precision", ctypes.c_int), ("cfl", ctypes.c_double), ("pfloor", ctypes.c_double)]


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
    L.mhd_floor_count.argtypes = [vp]
    L.mhd_floor_count.restype = ctypes.c_longlong
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
    L.mhd_init_batch.argtypes = [ip, ctypes.POINTER(Grid), ctypes.c_double, ctypes.POINTER(Scheme), vp,
                                 ctypes.POINTER(vp)]
    L.mhd_nbox.argtypes = [vp]
    L.mhd_nbox.restype = ip
    L.mhd_set_state_box.argtypes = [vp, ip, vp, vp, ip]
    L.mhd_get_state_box.argtypes = [vp, ip, vp, vp, ip]
    L.mhd_step_boxes.argtypes = [vp, dp]
    L.mhd_set_sweep_config.argtypes = [vp, ip, ip]
    L.mhd_get_sweep_config.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(ip)]
    L.mhd_autotune.argtypes = [vp, ip, ctypes.POINTER(ip), ctypes.POINTER(ip), dp]
    for name in ["mhd_init_batch", "mhd_set_state_box", "mhd_get_state_box", "mhd_step_boxes",
                 "mhd_set_sweep_config", "mhd_get_sweep_config", "mhd_autotune"]:
        getattr(L, name).restype = ctypes.c_int
    ll = ctypes.c_longlong
    fp = ctypes.c_void_p
    L.mhd_mlp_create.argtypes = [vp, ctypes.c_ulonglong, ctypes.POINTER(vp)]
    L.mhd_mlp_free.argtypes = [vp]
    L.mhd_mlp_free.restype = None
    L.mhd_mlp_nparam.argtypes = []
    L.mhd_mlp_nparam.restype = ip
    L.mhd_mlp_set_weights.argtypes = [vp, fp, ip]
    L.mhd_mlp_get_weights.argtypes = [vp, fp, ip]
    L.mhd_mlp_grad.argtypes = [vp, fp, fp, fp, ll, ctypes.c_double, fp, ctypes.POINTER(ctypes.c_float)]
    L.mhd_mlp_train_step.argtypes = [vp, fp, fp, fp, ll, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_float)]
    L.mhd_mlp_predict.argtypes = [vp, fp, ll, fp]
    L.mhd_nblocks.argtypes = [vp]
    L.mhd_nblocks.restype = ll
    L.mhd_block_features.argtypes = [vp, fp]
    L.mhd_block_error.argtypes = [vp, vp, fp]
    L.mhd_set_selector.argtypes = [vp, vp]
    L.mhd_selector_stats.argtypes = [vp, dp, dp]
    for name in ["mhd_mlp_create", "mhd_mlp_set_weights", "mhd_mlp_get_weights", "mhd_mlp_grad",
                 "mhd_mlp_train_step", "mhd_mlp_predict", "mhd_block_features", "mhd_block_error",
                 "mhd_set_selector", "mhd_selector_stats"]:
        getattr(L, name).restype = ctypes.c_int
    L.mhd_profile_begin.argtypes = [vp, ip]
    L.mhd_profile_end.argtypes = [vp, dp, ip, ctypes.POINTER(ctypes.c_int)]
    L.mhd_energies.argtypes = [vp, ctypes.c_double, dp]
    L.mhd_helicity.argtypes = [vp, dp]
    L.mhd_pressure_gradient.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp]
    L.mhd_set_sweep_pencils.argtypes = [vp, ip, ip]
    L.mhd_set_boundary.argtypes = [vp, ip]
    L.mhd_set_dirichlet.argtypes = [vp, ip, ip, dp, dp]
    L.mhd_get_dirichlet.argtypes = [vp, ip, ctypes.POINTER(ip)]
    L.mhd_get_boundary.argtypes = [vp, ctypes.POINTER(ip)]
    L.mhd_get_sweep_pencils.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(ip)]
    L.mhd_set_emf_staging.argtypes = [vp, ip]
    L.mhd_get_emf_staging.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(ip)]
    L.mhd_inject_wait_flag.argtypes = [vp, ctypes.c_uint]
    L.mhd_fma_peak.argtypes = [ip, ip, dp]
    # every entry point that returns an mhd_status; the others got their
    # restype above (long long, int, void, const char*)
    other = {"mhd_bad_cell", "mhd_clear_error", "mhd_device_bytes", "mhd_floor_count", "mhd_free",
             "mhd_last_error", "mhd_launches_per_step", "mhd_mlp_free", "mhd_mlp_nparam", "mhd_nblocks",
             "mhd_nbox"}
    for name in EXPORTS:
        if name not in other:
            getattr(L, name).restype = ctypes.c_int
    L.mhd_launches_per_step.restype = ctypes.c_int
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


def step_noalloc(U, B, dx, dt, gamma=5.0 / 3.0, recon="plm", riemann="roe", stream=None, pfloor=0.0):
    """One FP64 VL step of a caller-owned device state (torch CUDA float64
    tensors U (5, nz, ny, nx) and B (3, nz, ny, nx)), in place, through
    mhd_step_noalloc: no device memory is allocated (the scratch is a fixed
    array inside the library, at most NOALLOC_MAX_CELLS cells).  Calls that
    overlap on the GPU share that array and race: serialise them."""
    nz, ny, nx = U.shape[1:]
    g = Grid(nx, ny, nz, dx)
    s = Scheme(INTEGRATORS["vl"], RECONS[recon], SOLVERS[riemann], PRECISIONS["fp64"], 0.3, pfloor)
    pu, du = _ptr(U)
    pb, db = _ptr(B)
    if not (du and db):
        raise MHDError(MHD_EINVAL, "step_noalloc takes device arrays")
    st = lib().mhd_step_noalloc(ctypes.byref(g), gamma, ctypes.byref(s), dt, ctypes.c_void_p(pu),
                                ctypes.c_void_p(pb), ctypes.c_void_p(stream or 0))
    if st != MHD_OK:
        raise MHDError(st, lib().mhd_last_error(None).decode())


def fma_peak(precision="fp32", reps=5):
    """measured FMA throughput of the current device in TFLOP/s (mhd_fma_peak)"""
    out = ctypes.c_double()
    st = lib().mhd_fma_peak(PRECISIONS[precision], reps, ctypes.byref(out))
    if st != MHD_OK:
        raise MHDError(st, "mhd_fma_peak failed")
    return out.value


class Solver:
    """Periodic boxes advanced by the library (one mhd_ctx).  `shape` is one
    box (nz, ny, nx); `shapes` a list of boxes for a batch (each (nz, ny, nx),
    all with the same dx unless `dxs` is given)."""

    def __init__(self, shape, dx, gamma=5.0 / 3.0, integrator="vl", recon="plm", riemann="roe",
                 precision="fp64", cfl=0.3, stream=None, shapes=None, dxs=None, pfloor=0.0):
        shapes = [tuple(shape[-3:])] if shapes is None else [tuple(x) for x in shapes]
        dxs = [dx] * len(shapes) if dxs is None else list(dxs)
        self.shapes = shapes
        self.nbox = len(shapes)
        self.nz, self.ny, self.nx = shapes[0]
        self.precision = precision
        self.dtype = np.float32 if precision == "fp32" else np.float64
        grids = (Grid * self.nbox)(*[Grid(sh[2], sh[1], sh[0], d) for sh, d in zip(shapes, dxs)])
        s = Scheme(INTEGRATORS[integrator], RECONS[recon], SOLVERS[riemann], PRECISIONS[precision], cfl, pfloor)
        h = ctypes.c_void_p()
        st = lib().mhd_init_batch(self.nbox, grids, gamma, ctypes.byref(s), ctypes.c_void_p(stream or 0),
                                  ctypes.byref(h))
        if st != MHD_OK:
            raise MHDError(st, lib().mhd_last_error(None).decode())
        self.h = h
        self.n = self.nx * self.ny * self.nz

    def _check(self, st):
        if st != MHD_OK:
            raise MHDError(st, lib().mhd_last_error(self.h).decode())

    def set_state(self, U, B, box=0):
        pu, du = _ptr(U)
        pb, db = _ptr(B)
        assert du == db
        self._check(lib().mhd_set_state_box(self.h, box, ctypes.c_void_p(pu), ctypes.c_void_p(pb), du))

    def get_state(self, U=None, B=None, box=0):
        if U is None:
            nz, ny, nx = self.shapes[box]
            U = np.empty((5, nz, ny, nx), self.dtype)
            B = np.empty((3, nz, ny, nx), self.dtype)
        pu, du = _ptr(U)
        pb, db = _ptr(B)
        self._check(lib().mhd_get_state_box(self.h, box, ctypes.c_void_p(pu), ctypes.c_void_p(pb), du))
        return U, B

    def cfl_dts(self):
        dt = (ctypes.c_double * self.nbox)()
        self._check(lib().mhd_cfl_dt(self.h, dt))
        return np.array(dt[:])

    def cfl_dt(self):
        return float(self.cfl_dts()[0])

    def step(self, dt):
        if np.ndim(dt) == 0:
            self._check(lib().mhd_step(self.h, float(dt)))
        else:
            arr = (ctypes.c_double * self.nbox)(*[float(x) for x in dt])
            self._check(lib().mhd_step_boxes(self.h, arr))

    def advance(self, nsteps, use_graph=False):
        self._check(lib().mhd_advance(self.h, nsteps, int(use_graph)))

    def last_dts(self):
        dt = (ctypes.c_double * self.nbox)()
        self._check(lib().mhd_last_dt(self.h, dt))
        return np.array(dt[:])

    def last_dt(self):
        return float(self.last_dts()[0])

    def divBs(self):
        m = (ctypes.c_double * self.nbox)()
        r = (ctypes.c_double * self.nbox)()
        self._check(lib().mhd_divB(self.h, m, r))
        return np.array(m[:]), np.array(r[:])

    def divB(self):
        m, r = self.divBs()
        return float(m[0]), float(r[0])

    def sums_boxes(self):
        out = (ctypes.c_double * (8 * self.nbox))()
        self._check(lib().mhd_sums(self.h, out))
        return np.array(out[:]).reshape(self.nbox, 8)

    def sums(self):
        return self.sums_boxes()[0]

    def energies_boxes(self, jb_threshold=1.0):
        """per box: E_T, U_B, U_V, max dx|J|/|B|, cells above jb_threshold, max |J|"""
        out = (ctypes.c_double * (6 * self.nbox))()
        self._check(lib().mhd_energies(self.h, ctypes.c_double(jb_threshold), out))
        return np.array(out[:]).reshape(self.nbox, 6)

    def helicities(self):
        """magnetic helicity of every box (cuFFT, Coulomb gauge)"""
        out = (ctypes.c_double * self.nbox)()
        self._check(lib().mhd_helicity(self.h, out))
        return np.array(out[:])

    def helicity(self):
        return float(self.helicities()[0])

    def energies(self, jb_threshold=1.0):
        e = self.energies_boxes(jb_threshold)[0]
        return dict(E_T=e[0], U_B=e[1], U_V=e[2], jb_max=e[3], n_above=int(e[4]), j_max=e[5])

    def pressure_gradient_boxes(self, scale, thr, nlev=3):
        """per box: max of scale |grad P| / P, then the cells above thr * 2^l, l < nlev"""
        out = (ctypes.c_double * ((nlev + 1) * self.nbox))()
        self._check(lib().mhd_pressure_gradient(self.h, ctypes.c_double(scale), ctypes.c_double(thr), nlev, out))
        return np.array(out[:]).reshape(self.nbox, nlev + 1)

    def pressure_gradient(self, scale, thr, nlev=3):
        r = self.pressure_gradient_boxes(scale, thr, nlev)[0]
        return dict(max=float(r[0]), counts=[int(x) for x in r[1:]])

    def set_sweep_config(self, tile_len, blocks_per_sm):
        self._check(lib().mhd_set_sweep_config(self.h, tile_len, blocks_per_sm))

    def set_boundary(self, outflow_mask):
        """outflow (zero-gradient) boundaries on the axes of outflow_mask (bit d: axis d)"""
        self._check(lib().mhd_set_boundary(self.h, outflow_mask))

    def set_dirichlet(self, axis, nlayers, w_lo=None, w_hi=None):
        """Dirichlet sides along axis: nlayers ghost layers at each end held at
        w_lo / w_hi = (rho, vx, vy, vz, P, Bx, By, Bz); nlayers = 0 removes them"""
        lo = (ctypes.c_double * 8)(*([0.0] * 8 if w_lo is None else [float(v) for v in w_lo]))
        hi = (ctypes.c_double * 8)(*([0.0] * 8 if w_hi is None else [float(v) for v in w_hi]))
        self._check(lib().mhd_set_dirichlet(self.h, axis, nlayers, lo, hi))

    def dirichlet(self, axis):
        a = ctypes.c_int()
        self._check(lib().mhd_get_dirichlet(self.h, axis, ctypes.byref(a)))
        return a.value

    def boundary(self):
        a = ctypes.c_int()
        self._check(lib().mhd_get_boundary(self.h, ctypes.byref(a)))
        return a.value

    def set_sweep_pencils(self, pencil_mask, pencil_len=16):
        """VL face sweeps by pencils on the axes of pencil_mask (bit d: axis d)"""
        self._check(lib().mhd_set_sweep_pencils(self.h, pencil_mask, pencil_len))

    def sweep_pencils(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        self._check(lib().mhd_get_sweep_pencils(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def set_emf_staging(self, mode):
        """edge fields fused with the update that uses them (2, periodic
        boxes), a separate kernel whose planes are staged by the tensor
        memory accelerator (1, where the context allows it) or by per-thread
        loads (0, the default)"""
        self._check(lib().mhd_set_emf_staging(self.h, mode))

    def emf_staging(self):
        """(requested mode, form in use: 0 per-thread loads, 1 tensor copies, 2 fused)"""
        a, b = ctypes.c_int(), ctypes.c_int()
        self._check(lib().mhd_get_emf_staging(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def sweep_config(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        self._check(lib().mhd_get_sweep_config(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def autotune(self, reps=2):
        """time every sweep tiling on this batch, keep the fastest;
        returns (tile_len, blocks_per_sm, ms per step)"""
        a, b, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._check(lib().mhd_autotune(self.h, reps, ctypes.byref(a), ctypes.byref(b), ctypes.byref(ms)))
        return a.value, b.value, ms.value

    def sync(self):
        self._check(lib().mhd_sync(self.h))

    def floor_count(self):
        return int(lib().mhd_floor_count(self.h))

    def bad_cell(self):
        return lib().mhd_bad_cell(self.h)

    def inject_wait_flag(self, bits=1):
        """Test hook: set the device wait flag from the host, as a bounded
        device wait that gave up would (see mhd_inject_wait_flag)."""
        self._check(lib().mhd_inject_wait_flag(self.h, bits))

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
        ms = (ctypes.c_double * len(GROUPS))()
        steps = ctypes.c_int()
        self._check(lib().mhd_profile_end(self.h, ms, len(GROUPS), ctypes.byref(steps)))
        return dict(zip(GROUPS, ms[:])), steps.value

    # --- learned path selector -------------------------------------------
    def nblocks(self):
        return int(lib().mhd_nblocks(self.h))

    def block_features(self, out=None):
        """features of every 4^3 block of the current state (torch CUDA [nblocks, 48])"""
        import torch
        if out is None:
            out = torch.empty((self.nblocks(), 48), dtype=torch.float32, device="cuda")
        st = lib().mhd_block_features(self.h, ctypes.c_void_p(out.data_ptr()))
        if st != MHD_OK:
            raise MHDError(st, lib().mhd_last_error(None).decode())
        return out

    def set_selector(self, mlp):
        self._check(lib().mhd_set_selector(self.h, mlp.h if mlp is not None else None))
        self._selector = mlp

    def selector_stats(self):
        """fractions of 4^3 blocks and of sweep tiles the last step ran cheap"""
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(lib().mhd_selector_stats(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def free(self):
        if getattr(self, "h", None):
            lib().mhd_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def block_error(a, b, out=None):
    """per 4^3 block, max over the stored fields of mean |a - b| / scale (torch CUDA)"""
    import torch
    if out is None:
        out = torch.empty(a.nblocks(), dtype=torch.float32, device="cuda")
    st = lib().mhd_block_error(a.h, b.h, ctypes.c_void_p(out.data_ptr()))
    if st != MHD_OK:
        raise MHDError(st, lib().mhd_last_error(None).decode())
    return out


class MLP:
    """The selector network 48 -> 64 -> 64 -> 1 (BF16 tensor-core kernels).
    Parameters are packed FP32: W1[48][64], b1[64], W2[64][64], b2[64], w3[64], b3."""

    def __init__(self, seed=0, stream=None):
        h = ctypes.c_void_p()
        st = lib().mhd_mlp_create(ctypes.c_void_p(stream or 0), seed, ctypes.byref(h))
        if st != MHD_OK:
            raise MHDError(st, lib().mhd_last_error(None).decode())
        self.h = h
        self.nparam = int(lib().mhd_mlp_nparam())

    def set_weights(self, w):
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float32))
        assert w.size == self.nparam
        st = lib().mhd_mlp_set_weights(self.h, ctypes.c_void_p(w.ctypes.data), 0)
        if st != MHD_OK:
            raise MHDError(st, "mhd_mlp_set_weights")

    def weights(self):
        w = np.empty(self.nparam, np.float32)
        st = lib().mhd_mlp_get_weights(self.h, ctypes.c_void_p(w.ctypes.data), 0)
        if st != MHD_OK:
            raise MHDError(st, "mhd_mlp_get_weights")
        return w

    @staticmethod
    def _ptr(t):
        return ctypes.c_void_p(t.data_ptr()) if t is not None else None

    def grad(self, X, y, wgt=None):
        """gradient of the weighted mean BCE loss (torch CUDA tensors in and out)"""
        import torch
        g = torch.empty(self.nparam, dtype=torch.float32, device="cuda")
        loss = ctypes.c_float()
        wsum = float(wgt.sum().item()) if wgt is not None else float(X.shape[0])
        st = lib().mhd_mlp_grad(self.h, self._ptr(X), self._ptr(y), self._ptr(wgt), X.shape[0], wsum,
                                self._ptr(g), ctypes.byref(loss))
        if st != MHD_OK:
            raise MHDError(st, "mhd_mlp_grad")
        return g, loss.value

    def train_step(self, X, y, wgt=None, lr=1e-3, want_loss=False):
        loss = ctypes.c_float()
        wsum = float(wgt.sum().item()) if wgt is not None else float(X.shape[0])
        st = lib().mhd_mlp_train_step(self.h, self._ptr(X), self._ptr(y), self._ptr(wgt), X.shape[0], wsum, lr,
                                      ctypes.byref(loss) if want_loss else None)
        if st != MHD_OK:
            raise MHDError(st, "mhd_mlp_train_step")
        return loss.value if want_loss else None

    def predict(self, X):
        import torch
        out = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
        st = lib().mhd_mlp_predict(self.h, self._ptr(X), X.shape[0], self._ptr(out))
        if st != MHD_OK:
            raise MHDError(st, "mhd_mlp_predict")
        return out

    def free(self):
        if getattr(self, "h", None):
            lib().mhd_mlp_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
