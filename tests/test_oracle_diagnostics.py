"""Pins of the oracle's diagnostics (Sec. 4.3 and 4.5): the edge current
density of the discrete ABC field against its closed form, the face-based
magnetic energy U_B against (A^2+B^2+C^2) L^3/2 sinc^2(k dx/2), the flow and
total energies of a uniform drift, and the |J|/|B| refinement test of the
force-free field (|J|/|B| = k up to O((k dx)^2))."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1804_03479_b300 import inputs as I


def sinc(u):
    return math.sin(u) / u


@pytest.mark.parametrize("n,kmult", [(16, 1), (24, 2)])
def test_abc_edge_current_closed_form(n, kmult):
    # area-averaged face B of the ABC field: dx J_edge = 2 sin(k dx/2) sinc(k dx/2) B(edge point)
    st = I.abc(n, kmult=kmult, beta=1.0, noise=0.0)
    k, a, dx = st.meta["k"], st.meta["A"], st.dx
    J = orc.edge_current(st.B)
    fac = 2.0 * math.sin(0.5 * k * dx) * sinc(0.5 * k * dx)
    c = (np.arange(n) + 0.5) * dx          # cell centres
    f = np.arange(n) * dx                  # lower faces
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    zf, yf, xf = np.meshgrid(f, f, f, indexing="ij")
    # J_x at (x_i, y_{j-1/2}, z_{k-1/2}), J_y at (x_{i-1/2}, y_j, z_{k-1/2}), J_z at (x_{i-1/2}, y_{j-1/2}, z_k)
    Bx = a * np.sin(k * zf) + a * np.cos(k * yf)
    By = a * np.sin(k * xf) + a * np.cos(k * zf)
    Bz = a * np.sin(k * yf) + a * np.cos(k * xf)
    assert np.max(np.abs(J[0] - fac * Bx)) <= 1e-13
    assert np.max(np.abs(J[1] - fac * By)) <= 1e-13
    assert np.max(np.abs(J[2] - fac * Bz)) <= 1e-13


@pytest.mark.parametrize("n,kmult", [(16, 1), (32, 2)])
def test_abc_magnetic_energy_closed_form(n, kmult):
    st = I.abc(n, kmult=kmult, beta=1.0, noise=0.0)
    k, a, dx = st.meta["k"], st.meta["A"], st.dx
    d = orc.energies(st.U, st.B, dx, 1.0)
    ub = 3 * a * a / 2.0 * sinc(0.5 * k * dx) ** 2
    assert abs(d["U_B"] - ub) <= 1e-13 * ub
    assert d["U_V"] == 0.0


def test_uniform_drift_energies():
    st = I.abc(16, kmult=1, beta=0.7, noise=0.0, drift=(0.3, -0.2, 0.5), rho0=1.7)
    d = orc.energies(st.U, st.B, st.dx, 1.0)
    uv = 0.5 * 1.7 * (0.09 + 0.04 + 0.25)
    assert abs(d["U_V"] - uv) <= 1e-13 * uv
    P0 = st.meta["P0"]
    et = P0 / (st.gamma - 1.0) + uv + d["U_B"]      # the face-based U_B equals the cell-average sum only on average
    # e carries the cell-centred magnetic energy; the two differ at O((k dx)^2)
    assert abs(d["E_T"] - et) <= 0.05 * d["U_B"]
    assert abs(d["E_T"] - float(st.U[4].sum()) * st.dx ** 3) <= 1e-13 * d["E_T"]


def test_force_free_refinement_ratio():
    n, kmult = 32, 1
    st = I.abc(n, kmult=kmult, beta=1.0, noise=0.0)
    kdx = st.meta["k"] * st.dx
    d = orc.energies(st.U, st.B, st.dx, 0.9 * kdx)
    assert abs(d["jb_max"] / kdx - 1.0) <= 0.5 * kdx ** 2
    assert d["n_above"] == n ** 3
    assert orc.energies(st.U, st.B, st.dx, 1.1 * kdx)["n_above"] == 0
    # max |J| ~ k max |B| (|B| <= sqrt(3) * 2 a... bounded by k * max|B_cc|)
    W = orc.prim(st.U, st.B, st.gamma)
    bmax = float(np.sqrt(W[5] ** 2 + W[6] ** 2 + W[7] ** 2).max())
    assert d["j_max"] <= st.meta["k"] * bmax * 1.001


@pytest.mark.parametrize("n,kmult", [(16, 1), (24, 2), (32, 3)])
def test_abc_helicity_closed_form(n, kmult):
    """H = (A^2+B^2+C^2) L^4 / (2 pi n) (Sec. 4.5) for the ABC field; the
    cell-centre field of the discrete state is sinc(k dx/2) times the point
    field, so the discrete helicity carries sinc^2"""
    st = I.abc(n, kmult=kmult, beta=1.0, noise=0.0)
    k, a, dx = st.meta["k"], st.meta["A"], st.dx
    h = orc.helicity(st.B, dx)
    want = 3 * a * a / (2 * math.pi * kmult) * sinc(0.5 * k * dx) ** 2
    assert abs(h - want) <= 1e-12 * want
    # U_B = H k / 2 for the force-free state (both carry sinc^2)
    assert abs(orc.energies(st.U, st.B, dx, 1.0)["U_B"] - 0.5 * k * h) <= 1e-12 * h * k


def test_helicity_of_plane_polarised_and_mean_fields_is_zero():
    n = 16
    dx = 1.0 / n
    st = I.uniform(n)                                   # uniform B: the mean field has no potential
    assert abs(orc.helicity(st.B, dx)) <= 1e-15
    xf = np.arange(n) * dx
    B = np.zeros((3, n, n, n))
    B[1] = np.sin(2 * np.pi * (xf + 0.5 * dx))[None, None, :] * np.ones((n, n, 1))   # By(x): linear polarisation
    assert abs(orc.helicity(B, dx)) <= 1e-15
    # a circularly polarised wave (By, Bz) = (cos kx, sin kx) has H = -/+ L^3 / k
    c = (np.arange(n) + 0.5) * dx
    k = 2 * np.pi
    Bc = np.zeros((3, n, n, n))
    Bc[1] = np.cos(k * c)[None, None, :]
    Bc[2] = np.sin(k * c)[None, None, :]
    # faces hold the same values (By, Bz do not vary along y, z)
    h = orc.helicity(Bc, dx)
    assert abs(abs(h) - 1.0 / k) <= 1e-12


def _static_state(P, shape, dx, gam=5.0 / 3.0, Bv=(0.3, -0.2, 0.5), rho=1.0):
    nx, ny, nz = shape
    shp = (nz, ny, nx)
    Bf = np.stack([np.full(shp, b) for b in Bv])
    z = np.zeros(shp)
    U = I.conserved(np.full(shp, rho), z, z, z, P, Bf, gam)
    return U, np.ascontiguousarray(Bf), gam


def test_pressure_gradient_of_sines_closed_form():
    """P = P0 + sum_d a_d sin(k_d x_d + phi_d): the centred difference over
    2 dx is a_d cos(k_d x_d + phi_d) sin(k_d dx) / dx exactly"""
    shape = (24, 20, 16)
    dx = 1.0 / 24
    x = (np.arange(24) + 0.5) * dx
    y = (np.arange(20) + 0.5) * dx
    z = (np.arange(16) + 0.5) * dx
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    k = [2 * np.pi, 2 * np.pi * 24 / 20 * 2, 2 * np.pi * 24 / 16]   # whole periods on each side
    a = [0.2, 0.07, 0.11]
    ph = [0.3, 1.1, -0.4]
    P0 = 1.0
    P = P0 + a[0] * np.sin(k[0] * X + ph[0]) + a[1] * np.sin(k[1] * Y + ph[1]) + a[2] * np.sin(k[2] * Z + ph[2])
    U, Bf, gam = _static_state(P, shape, dx)
    gx = a[0] * np.cos(k[0] * X + ph[0]) * np.sin(k[0] * dx) / dx
    gy = a[1] * np.cos(k[1] * Y + ph[1]) * np.sin(k[1] * dx) / dx
    gz = a[2] * np.cos(k[2] * Z + ph[2]) * np.sin(k[2] * dx) / dx
    scale = 0.05
    want = scale * np.sqrt(gx ** 2 + gy ** 2 + gz ** 2) / P
    thr = 0.04
    r = orc.pressure_gradient(U, Bf, dx, gam, scale, thr, nlev=3)
    assert np.max(np.abs(r["score"] - want)) <= 1e-12 * want.max()
    assert abs(r["max"] - want.max()) <= 1e-12 * want.max()
    for l in range(3):
        t = thr * 2.0 ** l
        assert np.min(np.abs(want - t)) > 1e-9          # no cell sits on a threshold
        assert r["counts"][l] == int(np.count_nonzero(want > t))
    assert r["counts"][0] > r["counts"][1] > 0


def test_pressure_gradient_outflow_ramp():
    """P linear in x with outflow along x: the interior centred difference is
    the slope, the two end cells see half of it (their outer neighbour is
    the cell itself); y and z periodic and uniform contribute nothing"""
    shape = (12, 4, 4)
    dx = 1.0 / 12
    x = (np.arange(12) + 0.5) * dx
    P = np.broadcast_to(0.5 + 2.0 * x, (4, 4, 12)).copy()
    U, Bf, gam = _static_state(P, shape, dx)
    r = orc.pressure_gradient(U, Bf, dx, gam, 1.0, 1.0, nlev=2, bc=1)
    want = 2.0 / P
    want[:, :, 0] *= 0.5
    want[:, :, -1] *= 0.5
    assert np.max(np.abs(r["score"] - want)) <= 1e-12
    # periodic along x: the wrap turns the ends into a jump of -2 over 2 dx
    rp = orc.pressure_gradient(U, Bf, dx, gam, 1.0, 1.0, nlev=2, bc=0)
    jump = (P[:, :, 0] - P[:, :, -2]) * (0.5 / dx) / P[:, :, -1]
    assert np.max(np.abs(rp["score"][:, :, -1] - np.abs(jump))) <= 1e-12


def test_pressure_gradient_uniform_and_scale_free():
    shape = (8, 8, 8)
    dx = 1.0 / 8
    U, Bf, gam = _static_state(np.full((8, 8, 8), 0.7), shape, dx)
    r = orc.pressure_gradient(U, Bf, dx, gam, 100.0 * 0.05, 1.25, nlev=3)
    assert r["max"] < 1e-12 and r["counts"] == [0, 0, 0]
    # blast state: the score does not depend on the unit of pressure
    st = I.mhd_blast(24, r0=0.1)
    a = orc.pressure_gradient(st.U, st.B, st.dx, st.gamma, 10.0, 1.25)
    U2 = st.U.copy()
    U2[1:4] *= np.sqrt(3.0)         # M scales with v ~ sqrt(P / rho) at fixed rho
    U2[4] *= 3.0
    b = orc.pressure_gradient(U2, st.B * np.sqrt(3.0), st.dx, st.gamma, 10.0, 1.25)
    assert np.max(np.abs(a["score"] - b["score"])) <= 1e-12 * a["max"]
    assert a["counts"] == b["counts"] and a["counts"][0] > 0
