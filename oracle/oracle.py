"""ctypes binding of the FP64 CPU oracle (``mhd_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by
the CPU-baseline leg of the benchmark.  The product path never imports it.

Layout of the arrays passed in and out (float64, C order):
  U: (5, nz, ny, nx)  rho, Mx, My, Mz, e   (cell averages, Eq. 11)
  B: (3, nz, ny, nx)  Bx at x_{i-1/2}, By at y_{j-1/2}, Bz at z_{k-1/2} (Eq. 14)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhd_oracle.c")
_LIB = os.path.join(_HERE, "libmhd_oracle.so")

VL, CTU = 0, 1
PLM, PPM, PLM_PRIM = 0, 1, 2
ROE, HLLD, HLLE = 0, 1, 2

INTEGRATORS = {"vl": VL, "ctu": CTU}
RECONS = {"plm": PLM, "ppm": PPM, "plm_prim": PLM_PRIM}
SOLVERS = {"roe": ROE, "hlld": HLLD, "hlle": HLLE}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-ffp-contract=off: no fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_step.restype = ctypes.c_long
        L.orc_step.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [ctypes.c_int] * 3 + \
                              [ctypes.c_double, dp, dp]
        L.orc_step_floor.restype = ctypes.c_long
        L.orc_step_floor.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [ctypes.c_int] * 3 + \
                                    [ctypes.c_double, ctypes.c_double, dp, dp, ctypes.POINTER(ctypes.c_long)]
        L.orc_cfl_dt_floor.restype = ctypes.c_double
        L.orc_cfl_dt_floor.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 4 + [dp, dp]
        L.orc_step_full.restype = ctypes.c_long
        L.orc_step_full.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [ctypes.c_int] * 3 + \
                                   [ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp, ctypes.POINTER(ctypes.c_long)]
        L.orc_cfl_dt_full.restype = ctypes.c_double
        L.orc_cfl_dt_full.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 4 + [ctypes.c_int, dp, dp]
        L.orc_divB_bc.restype = None
        L.orc_divB_bc.argtypes = [ctypes.c_int] * 4 + [dp, dp, dp]
        L.orc_prim_bc.restype = None
        L.orc_prim_bc.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double, ctypes.c_int, dp, dp, dp]
        L.orc_cfl_dt.restype = ctypes.c_double
        L.orc_cfl_dt.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [dp, dp]
        L.orc_divB.restype = None
        L.orc_divB.argtypes = [ctypes.c_int] * 3 + [dp, dp, dp]
        L.orc_sums.restype = None
        L.orc_sums.argtypes = [ctypes.c_int] * 3 + [dp, dp, dp]
        L.orc_prim.restype = None
        L.orc_prim.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double, dp, dp, dp]
        L.orc_eigen.restype = None
        L.orc_eigen.argtypes = [dp, ctypes.c_double, ctypes.c_double, dp, dp, dp]
        L.orc_riemann.restype = ctypes.c_int
        L.orc_riemann.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double, dp]
        L.orc_hlld_fan.restype = None
        L.orc_hlld_fan.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_hlle_fan.restype = None
        L.orc_hlle_fan.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_roe_waves.restype = ctypes.c_int
        L.orc_roe_waves.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, dp, dp, dp]
        L.orc_flux_phys.restype = None
        L.orc_flux_phys.argtypes = [dp, ctypes.c_double, ctypes.c_double, dp]
        L.orc_recon_cell.restype = None
        L.orc_recon_cell.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_edge_current.restype = None
        L.orc_edge_current.argtypes = [ctypes.c_int] * 3 + [dp, dp]
        L.orc_energies.restype = None
        L.orc_energies.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double, dp, dp, ctypes.c_double, dp]
        L.orc_set_threads.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def set_threads(n: int) -> int:
    """OpenMP threads of the oracle's loops (n <= 0: leave as is); returns
    the count in effect."""
    return int(lib().orc_set_threads(int(n)))


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def step(U: np.ndarray, B: np.ndarray, dx: float, gamma: float, dt: float,
         integrator="vl", recon="plm", riemann="roe") -> int:
    """Advance (U, B) in place by dt; returns the count of Roe->HLLE fallbacks."""
    nz, ny, nx = U.shape[1:]
    assert U.shape == (5, nz, ny, nx) and B.shape == (3, nz, ny, nx)
    return int(lib().orc_step(nx, ny, nz, dx, gamma, INTEGRATORS[integrator], RECONS[recon],
                              SOLVERS[riemann], dt, _p(U), _p(B)))


def step_floor(U: np.ndarray, B: np.ndarray, dx: float, gamma: float, dt: float,
               integrator="vl", recon="plm", riemann="roe", pfloor=0.0) -> tuple[int, int]:
    """step() with a pressure floor: cells whose P falls below pfloor at the
    start of the step get their energy raised to P = pfloor, and every
    primitive pass uses max(P, pfloor).  Returns (Roe->HLLE fallbacks,
    floored cells)."""
    nz, ny, nx = U.shape[1:]
    assert U.shape == (5, nz, ny, nx) and B.shape == (3, nz, ny, nx)
    nf = ctypes.c_long(0)
    fb = lib().orc_step_floor(nx, ny, nz, dx, gamma, INTEGRATORS[integrator], RECONS[recon], SOLVERS[riemann],
                              dt, pfloor, _p(U), _p(B), ctypes.byref(nf))
    return int(fb), int(nf.value)


def step_bc(U: np.ndarray, B: np.ndarray, dx: float, gamma: float, dt: float,
            integrator="vl", recon="plm", riemann="roe", bc=0, pfloor=0.0) -> int:
    """step() with outflow (zero-gradient) boundaries along the axes of the
    bit mask bc (bit d: axis d) and periodic ones elsewhere, VL or CTU.
    Returns the Roe->HLLE fallbacks."""
    nz, ny, nx = U.shape[1:]
    assert U.shape == (5, nz, ny, nx) and B.shape == (3, nz, ny, nx)
    nf = ctypes.c_long(0)
    r = lib().orc_step_full(nx, ny, nz, dx, gamma, INTEGRATORS[integrator], RECONS[recon], SOLVERS[riemann],
                            dt, pfloor, bc, _p(U), _p(B), ctypes.byref(nf))
    return int(r)


def fix_layers(U, B, gamma, axis, nl, wlo, whi):
    """Dirichlet sides (the shock tubes of Sec. 5.1 hold the left and right
    states at the ends of the box): the nl outermost cells at each end of
    `axis` are ghost cells kept at a fixed state, written here in place.
    w = (rho, vx, vy, vz, P, Bx, By, Bz) in box axes; a ghost cell gets the
    conserved state of w and its three lower faces the field of w, except
    the lower face along `axis` of the first upper ghost cell, which is the
    upper boundary face of the interior (advanced by CT like every interior
    face).  Cells and faces beyond the box continue the last ones (the
    outflow rule).  With nl >= 2 (VL with PPM: 3) the interior sees an
    unbounded region of the fixed state (more layers change nothing): only
    the first ghost cell's state moves within a step, and in VL PPM reads the
    half-step states one cell further than the PLM slope."""
    nd = U.shape[3 - axis]
    assert nd >= 2 * nl + 1

    def layer(sl):
        idx = [slice(None)] * 3
        idx[2 - axis] = sl
        return tuple(idx)

    for w, sl in ((wlo, slice(0, nl)), (whi, slice(nd - nl, nd))):
        rho, v, P, b = w[0], np.asarray(w[1:4], float), w[4], np.asarray(w[5:8], float)
        e = P / (gamma - 1.0) + 0.5 * rho * float(v @ v) + 0.5 * float(b @ b)
        for f, val in enumerate((rho, rho * v[0], rho * v[1], rho * v[2], e)):
            U[f][layer(sl)] = val
        for m in range(3):
            if m == axis and sl.start == nd - nl:
                B[m][layer(slice(nd - nl + 1, nd))] = b[m]      # keep the interior's upper face
            else:
                B[m][layer(sl)] = b[m]


def step_dirichlet(U, B, dx, gamma, dt, integrator, recon, riemann, axis, nl, wlo, whi, bc=0, pfloor=0.0) -> int:
    """One step with Dirichlet sides along `axis` (fix_layers), outflow
    clamping beyond them and the boundaries of the mask bc elsewhere; the
    ghost layers are put back to the fixed state after the step."""
    fb = step_bc(U, B, dx, gamma, dt, integrator, recon, riemann, bc=bc | (1 << axis), pfloor=pfloor)
    fix_layers(U, B, gamma, axis, nl, wlo, whi)
    return fb


def cfl_dt(U, B, dx, gamma, cfl, pfloor=0.0, bc=0) -> float:
    nz, ny, nx = U.shape[1:]
    if pfloor > 0.0 or bc:
        return float(lib().orc_cfl_dt_full(nx, ny, nz, dx, gamma, cfl, pfloor, bc, _p(U), _p(B)))
    return float(lib().orc_cfl_dt(nx, ny, nz, dx, gamma, cfl, _p(U), _p(B)))


def divB(B, bc=0) -> tuple[float, float]:
    """(max_c |sum_d dB_d| (= |div B| dx), B_rms); along an outflow axis the
    face beyond the last cell continues the last face."""
    nz, ny, nx = B.shape[1:]
    m = np.zeros(1); r = np.zeros(1)
    lib().orc_divB_bc(nx, ny, nz, bc, _p(B), _p(m), _p(r))
    return float(m[0]), float(r[0])


def sums(U, B) -> np.ndarray:
    nz, ny, nx = U.shape[1:]
    out = np.zeros(8)
    lib().orc_sums(nx, ny, nz, _p(U), _p(B), _p(out))
    return out


def prim(U, B, gamma, bc=0) -> np.ndarray:
    nz, ny, nx = U.shape[1:]
    W = np.zeros((8, nz, ny, nx))
    lib().orc_prim_bc(nx, ny, nz, gamma, bc, _p(U), _p(B), _p(W))
    return W


def eigen(w, bn, gamma):
    w = _f64(w); lam = np.zeros(7); R = np.zeros(49); L = np.zeros(49)
    lib().orc_eigen(_p(w), bn, gamma, _p(lam), _p(R), _p(L))
    return lam, R.reshape(7, 7), L.reshape(7, 7)


def riemann(solver, wl, wr, bn, gamma):
    wl = _f64(wl); wr = _f64(wr); f = np.zeros(7)
    fb = lib().orc_riemann(SOLVERS[solver], _p(wl), _p(wr), bn, gamma, _p(f))
    return f, int(fb)


def hlld_fan(wl, wr, bn, gamma):
    """HLLD fan: speeds (S_L, S*_L, S_M, S*_R, S_R) and the six conserved
    states (U_L, U*_L, U**_L, U**_R, U*_R, U_R), rows (rho, M_n, M_t1, M_t2,
    e, B_t1, B_t2)."""
    S = np.zeros(5); Uf = np.zeros((6, 7))
    lib().orc_hlld_fan(_p(_f64(wl)), _p(_f64(wr)), bn, gamma, _p(S), _p(Uf))
    return S, Uf


def hlle_fan(wl, wr, bn, gamma):
    """HLLE fan: Einfeldt speeds (S_L, S_R) and the HLL average state."""
    S = np.zeros(2); Uh = np.zeros(7)
    lib().orc_hlle_fan(_p(_f64(wl)), _p(_f64(wr)), bn, gamma, _p(S), _p(Uh))
    return S, Uh


def roe_waves(wl, wr, bn, gamma):
    wl = _f64(wl); wr = _f64(wr)
    lam = np.zeros(7); eta = np.zeros(7); ru = np.zeros(49)
    ok = lib().orc_roe_waves(_p(wl), _p(wr), bn, gamma, _p(lam), _p(eta), _p(ru))
    return bool(ok), lam, eta, ru.reshape(7, 7)


def flux_phys(w, bn, gamma):
    w = _f64(w); f = np.zeros(7)
    lib().orc_flux_phys(_p(w), bn, gamma, _p(f))
    return f


def recon_cell(recon, w5, bn5, gamma, trace=False, dtdx=0.0):
    w5 = _f64(w5).reshape(5, 7); bn5 = _f64(bn5)
    wm = np.zeros(7); wp = np.zeros(7)
    lib().orc_recon_cell(RECONS[recon], int(trace), _p(w5), _p(bn5), gamma, dtdx, _p(wm), _p(wp))
    return wm, wp


def edge_current(B) -> np.ndarray:
    """dx J on the cell edges (layout of the edge E fields)."""
    nz, ny, nx = B.shape[1:]
    J = np.zeros((3, nz, ny, nx))
    lib().orc_edge_current(nx, ny, nz, _p(B), _p(J))
    return J


def energies(U, B, dx, thr) -> dict:
    """E_T, U_B (face-based), U_V, max dx|J|/|B|, cells above thr, max |J|."""
    nz, ny, nx = U.shape[1:]
    out = np.zeros(6)
    lib().orc_energies(nx, ny, nz, dx, _p(U), _p(B), thr, _p(out))
    return dict(E_T=out[0], U_B=out[1], U_V=out[2], jb_max=out[3], n_above=int(out[4]), j_max=out[5])


def pressure_gradient(U, B, dx, gamma, scale, thr, nlev=3, bc=0) -> dict:
    """Refinement indicator of the magnetised blast run (Sec. 5.1): per cell
    the normalised pressure gradient scale * |grad P| / P (scale = 100 r0 in
    that run), grad P by centred differences of the cell pressure of prim()
    over 2 dx, a neighbour beyond an outflow side being the cell itself.
    Returns its maximum and, for l < nlev, the number of cells above
    thr * 2^l (the run refines to level n above 1.25 * 2^(n-1))."""
    P = prim(U, B, gamma, bc=bc)[4]
    g2 = np.zeros_like(P)
    for d in range(3):
        ax = 2 - d                                   # array order (z, y, x)
        n = P.shape[ax]
        if bc >> d & 1:
            up = np.take(P, np.minimum(np.arange(n) + 1, n - 1), axis=ax)
            dn = np.take(P, np.maximum(np.arange(n) - 1, 0), axis=ax)
        else:
            up = np.roll(P, -1, axis=ax)
            dn = np.roll(P, 1, axis=ax)
        g2 += (up - dn) ** 2
    score = scale * (np.sqrt(g2) * (0.5 / dx)) / P
    return dict(max=float(score.max()), counts=[int(np.count_nonzero(score > thr * 2.0 ** l)) for l in range(nlev)],
                score=score)


def helicity(B, dx) -> float:
    """Magnetic helicity H = sum A.B dx^3 (Sec. 4.5) of the cell-centre field
    (mean of the two faces per axis) on the periodic box: A in the Coulomb
    gauge from the discrete Fourier transform of B, A_k = i k x B_k / |k|^2,
    and H by Parseval, dx^3 / N sum_k Re(conj(A_k) . B_k); the k = 0 mode
    (the mean field) carries no A."""
    nz, ny, nx = B.shape[1:]
    bc = np.stack([0.5 * (B[0] + np.roll(B[0], -1, axis=2)),
                   0.5 * (B[1] + np.roll(B[1], -1, axis=1)),
                   0.5 * (B[2] + np.roll(B[2], -1, axis=0))])
    Bk = np.fft.fftn(bc, axes=(1, 2, 3))
    kx = 2 * np.pi * np.fft.fftfreq(nx, d=dx)
    ky = 2 * np.pi * np.fft.fftfreq(ny, d=dx)
    kz = 2 * np.pi * np.fft.fftfreq(nz, d=dx)
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    k2 = KX * KX + KY * KY + KZ * KZ
    k2[0, 0, 0] = 1.0
    cx = KY * Bk[2] - KZ * Bk[1]
    cy = KZ * Bk[0] - KX * Bk[2]
    cz = KX * Bk[1] - KY * Bk[0]
    Ak = 1j * np.stack([cx, cy, cz]) / k2
    Ak[:, 0, 0, 0] = 0.0
    n = nx * ny * nz
    return float(np.real(np.sum(np.conj(Ak) * Bk)) * dx ** 3 / n)
