"""Outflow (zero-gradient) boundaries of the oracle, VL and CTU integrators:
a face or cell beyond the last one along an outflow axis is the last one,
and the flux through the outer face of the last cell is the Riemann flux
between that cell and its copy (for CTU, of the cell's own upper and lower
traced states, corrected in the second stage).  Pinned by: periodic
behaviour unchanged for bc = 0; the B = 0 Sod tube against Toro's exact
Euler solution after its shock and rarefaction have left the box; a density
pulse carried out of the box leaving the uniform background; the discrete
divergence kept at its value."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1804_03479_b300 import inputs as I

from test_oracle_scheme import exact_euler


def tube_1d(n, wl, wr, g, x0=0.5, B=(0.0, 0.0, 0.0), m=1):
    dx = 1.0 / n
    x = (np.arange(n) + 0.5) * dx
    left = x < x0
    shp = (m, m, n)
    rho = np.broadcast_to(np.where(left, wl[0], wr[0]), shp).copy()
    u = np.broadcast_to(np.where(left, wl[1], wr[1]), shp).copy()
    P = np.broadcast_to(np.where(left, wl[2], wr[2]), shp).copy()
    z = np.zeros(shp)
    Bf = np.stack([np.full(shp, B[0]), np.full(shp, B[1]), np.full(shp, B[2])])
    return I.conserved(rho, u, z, z, P, Bf, g), np.ascontiguousarray(Bf), x, dx


@pytest.mark.parametrize("integ", ["vl", "ctu"])
def test_bc0_is_the_periodic_step(integ):
    st = I.abc(12, kmult=1, beta=0.5, seed=4, noise=2e-2)
    Ua, Ba = st.U.copy(), st.B.copy()
    Ub, Bb = st.U.copy(), st.B.copy()
    dt = orc.cfl_dt(Ua, Ba, st.dx, st.gamma, 0.3)
    orc.step(Ua, Ba, st.dx, st.gamma, dt, integ, "ppm", "hlld")
    orc.step_bc(Ub, Bb, st.dx, st.gamma, dt, integ, "ppm", "hlld", bc=0)
    assert np.array_equal(Ua, Ub) and np.array_equal(Ba, Bb)


@pytest.mark.parametrize("integ,recon,solver", [("vl", "plm", "roe"), ("vl", "ppm", "hlld"), ("vl", "plm", "hlle"),
                                               ("ctu", "plm", "roe"), ("ctu", "ppm", "roe"), ("ctu", "plm", "hlld")])
def test_sod_through_outflow_boundaries(integ, recon, solver):
    """the waves leave through both ends (T = 0.4); inside, the profile still
    converges to the exact solution of the unbounded problem"""
    g = 1.4
    wl, wr = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    T = 0.4

    def err(n):
        U, B, x, dx = tube_1d(n, wl, wr, g)
        t = 0.0
        while t < T:
            dt = min(orc.cfl_dt(U, B, dx, g, 0.4, bc=1), T - t)
            orc.step_bc(U, B, dx, g, dt, integ, recon, solver, bc=1)
            t += dt
        sel = (x > 0.1) & (x < 0.9)
        ex = exact_euler(wl, wr, g, (x[sel] - 0.5) / T)
        return np.abs(U[0, 0, 0, sel] - ex[:, 0]).mean()

    e128, e512 = err(128), err(512)
    assert e512 < 6e-3, e512
    assert e128 / e512 > 2.0


@pytest.mark.parametrize("integ", ["vl", "ctu"])
def test_pulse_leaves_the_box(integ):
    """a density pulse in a uniform flow (v = 1 along x, B along x) crosses the
    outflow boundary; the zero-gradient inflow keeps feeding the background,
    so once the pulse is out the box holds the uniform state again"""
    n, g = 128, 5.0 / 3.0
    dx = 1.0 / n
    x = (np.arange(n) + 0.5) * dx
    shp = (1, 1, n)
    rho = np.broadcast_to(1.0 + 0.2 * np.exp(-((x - 0.5) / 0.08) ** 2), shp).copy()
    u = np.ones(shp)
    z = np.zeros(shp)
    Bf = np.stack([np.full(shp, 0.3), z, z])
    U = I.conserved(rho, u, z, z, np.ones(shp), Bf, g)
    B = np.ascontiguousarray(Bf)
    t = 0.0
    while t < 1.2:
        dt = orc.cfl_dt(U, B, dx, g, 0.4, bc=1)
        orc.step_bc(U, B, dx, g, dt, integ, "ppm", "roe", bc=1)
        t += dt
    W = orc.prim(U, B, g, bc=1)
    assert np.abs(W[0] - 1.0).max() < 2e-3
    assert np.abs(W[1] - 1.0).max() < 2e-3


@pytest.mark.parametrize("integ", ["vl", "ctu"])
@pytest.mark.parametrize("bc", [1, 2, 4, 7])
def test_outflow_keeps_div_b(bc, integ):
    """a field without divergence under either boundary convention (B_x
    uniform, B_y(z), B_z(y)) with a noisy flow: CT keeps the discrete
    divergence at round-off in every cell, the boundary cells included"""
    n = 12
    st = I.abc(n, kmult=1, beta=1.0, seed=8, noise=5e-2)
    dx = st.dx
    c = (np.arange(n) + 0.5) * dx
    Bf = np.zeros((3, n, n, n))
    Bf[0] = 0.4
    Bf[1] = (0.3 * np.sin(2 * np.pi * c))[:, None, None] * np.ones((1, n, n))   # By(z)
    Bf[2] = (0.2 * np.cos(2 * np.pi * c))[None, :, None] * np.ones((n, 1, n))   # Bz(y)
    W = orc.prim(st.U, st.B, st.gamma)
    U = I.conserved(W[0], W[1], W[2], W[3], W[4], Bf, st.gamma)
    B = np.ascontiguousarray(Bf)
    m0, brms = orc.divB(B, bc=bc)
    assert m0 <= 1e-14 * brms
    for _ in range(5):
        dt = orc.cfl_dt(U, B, dx, st.gamma, 0.3, bc=bc)
        orc.step_bc(U, B, dx, st.gamma, dt, integ, "plm", "hlld", bc=bc)
    m, brms = orc.divB(B, bc=bc)
    assert m <= 1e-13 * brms


def test_ctu_outflow_open_box_positive_and_conservative_inside():
    """CTU with outflow on every axis: the smooth open-box state stays
    positive and the divergence stays at round-off"""
    st = I.open_box((16, 12, 10), seed=5)
    U, B = st.U.copy(), st.B.copy()
    for _ in range(3):
        dt = orc.cfl_dt(U, B, st.dx, st.gamma, 0.3, bc=7)
        orc.step_bc(U, B, st.dx, st.gamma, dt, "ctu", "ppm", "roe", bc=7)
    W = orc.prim(U, B, st.gamma, bc=7)
    assert W[0].min() > 0.3 and W[4].min() > 0.2
    m, brms = orc.divB(B, bc=7)
    assert m <= 1e-13 * brms
