"""Whole-step pins of the oracle (VL and CTU with CT, Sec. 3.2).

- a uniform state is a steady solution (any v, B);
- the discrete divergence of Eq. 16 does not change (Sec. 3.1: CT keeps it);
- mass, momentum, energy and the face-field sums are conserved (Eq. 10);
- the scheme commutes with a cyclic relabelling of the axes;
- linear waves converge at second order (Sec. 5.1 (i));
- the ABC force-free state stays static up to truncation error O(dx^2);
- with B = 0 a shock tube converges to Toro's exact Euler solution;
- the CFL step matches closed forms for simple states.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1804_03479_b300 import inputs as I

COMBOS = [(i, r, s) for i in ("vl", "ctu") for r in ("plm", "ppm") for s in ("roe", "hlld", "hlle")]


def advance(st, nsteps, integ, recon, solver, cfl=0.3, U=None, B=None):
    U = st.U.copy() if U is None else U
    B = st.B.copy() if B is None else B
    for _ in range(nsteps):
        dt = orc.cfl_dt(U, B, st.dx, st.gamma, cfl)
        orc.step(U, B, st.dx, st.gamma, dt, integ, recon, solver)
    return U, B


@pytest.mark.parametrize("integ,recon,solver", COMBOS + [("vl", "plm_prim", "hlle")])
def test_uniform_state_is_steady(integ, recon, solver):
    st = I.uniform(8, shape=(8, 6, 4))
    U, B = advance(st, 3, integ, recon, solver)
    assert np.abs(U - st.U).max() < 1e-14
    assert np.abs(B - st.B).max() < 1e-14


@pytest.mark.parametrize("integ,recon,solver", COMBOS + [("vl", "plm_prim", "hlle")])
def test_divergence_and_conservation(integ, recon, solver):
    st = I.abc(16, kmult=2, beta=0.5, seed=3, noise=1e-2)
    m0, brms = orc.divB(st.B)
    s0 = orc.sums(st.U, st.B)
    U, B = advance(st, 4, integ, recon, solver)
    m1, brms1 = orc.divB(B)
    assert m0 / brms < 1e-13 and m1 / brms1 < 1e-13
    s1 = orc.sums(U, B)
    scale = np.array([np.abs(st.U[f]).sum() for f in range(5)] + [np.abs(st.B[d]).sum() for d in range(3)])
    assert np.all(np.abs(s1 - s0) <= 1e-13 * scale + 1e-12)


def _cycle(st):
    """relabel the axes x' = y, y' = z, z' = x (a rotation of the box)."""
    T = lambda a: np.ascontiguousarray(np.transpose(a, (2, 0, 1)))
    U = np.stack([T(st.U[0]), T(st.U[2]), T(st.U[3]), T(st.U[1]), T(st.U[4])])
    B = np.stack([T(st.B[1]), T(st.B[2]), T(st.B[0])])
    return U, B


def _uncycle(U, B):
    T = lambda a: np.ascontiguousarray(np.transpose(a, (1, 2, 0)))
    Uo = np.stack([T(U[0]), T(U[3]), T(U[1]), T(U[2]), T(U[4])])
    Bo = np.stack([T(B[2]), T(B[0]), T(B[1])])
    return Uo, Bo


@pytest.mark.parametrize("integ,recon,solver", [("vl", "plm", "roe"), ("ctu", "ppm", "hlld"),
                                                ("ctu", "plm", "hlle"), ("vl", "ppm", "roe")])
def test_axis_relabelling_commutes(integ, recon, solver):
    # a non-cubic box, so the relabelled problem is a different array shape
    st = I.abc(None, kmult=1, beta=0.5, seed=4, noise=3e-2, shape=(8, 12, 16), L=1.0)
    dt = 0.2 * orc.cfl_dt(st.U, st.B, st.dx, st.gamma, 0.3)
    U1, B1 = st.U.copy(), st.B.copy()
    U2, B2 = _cycle(st)
    for _ in range(2):
        orc.step(U1, B1, st.dx, st.gamma, dt, integ, recon, solver)
        orc.step(U2, B2, st.dx, st.gamma, dt, integ, recon, solver)
    U2, B2 = _uncycle(U2, B2)
    assert np.abs(U2 - U1).max() < 1e-13 * np.abs(U1).max()
    assert np.abs(B2 - B1).max() < 1e-13 * np.abs(B1).max()


def l1_after_period(n, wave, integ, recon, solver, shape=None, direction=(1, 1, 1), cfl=0.3):
    st = I.linear_wave(n, wave, shape=shape, direction=direction)
    U, B = st.U.copy(), st.B.copy()
    T = st.meta["period"]; t = 0.0
    while t < T:
        dt = min(orc.cfl_dt(U, B, st.dx, st.gamma, cfl), T - t)
        orc.step(U, B, st.dx, st.gamma, dt, integ, recon, solver)
        t += dt
    W0 = orc.prim(st.U, st.B, st.gamma); W1 = orc.prim(U, B, st.gamma)
    # E_L1 of Sec. 5.1 (i), summed over the eight primitive variables
    return np.abs(W1 - W0).mean(axis=(1, 2, 3)).sum()


@pytest.mark.parametrize("wave", ["fast", "alfven", "slow"])
@pytest.mark.parametrize("integ", ["vl", "ctu"])
@pytest.mark.parametrize("recon", ["plm", "ppm"])
def test_linear_wave_second_order_3d(wave, integ, recon):
    """Diagonal linear waves, one period, Roe (Sec. 5.1 (i)): E_L1 ~ N^-2.
    PPM is still pre-asymptotic at N = 16 -> 32 (limiter clipping at the
    extrema), so its bound is looser; the 1-D test below pins its order."""
    e16 = l1_after_period(16, wave, integ, recon, "roe")
    e32 = l1_after_period(32, wave, integ, recon, "roe")
    assert e16 / e32 > (3.4 if recon == "plm" else 2.8)
    assert e32 < 1e-7   # amplitude 1e-6: the error is a small fraction of it


@pytest.mark.parametrize("integ,recon,solver", COMBOS)
def test_linear_wave_second_order_1d(integ, recon, solver):
    e = [l1_after_period(n, "fast", integ, recon, solver, shape=(n, 1, 1), direction=(1, 0, 0))
         for n in (64, 128, 256)]
    assert e[1] / e[2] > 3.5, e       # slope at least 1.8 on the finest pair
    assert e[0] / e[1] > 3.2, e


@pytest.mark.parametrize("integ,recon", [("vl", "plm"), ("ctu", "ppm")])
def test_abc_force_free_state_static(integ, recon):
    """The ABC field is force-free (Sec. 5.1 (v)): with no velocity noise the
    flow it drives in a fixed time is truncation error.  Its mean (the L1
    norm of Sec. 5.1 (i)) falls as dx^2; the maximum is set by the limiters'
    clipping at the field's extrema and falls more slowly."""
    def vmean(n):
        st = I.abc(n, kmult=1, beta=1.0, noise=0.0)
        U, B = st.U.copy(), st.B.copy()
        t, T = 0.0, 0.05
        while t < T:
            dt = min(orc.cfl_dt(U, B, st.dx, st.gamma, 0.3), T - t)
            orc.step(U, B, st.dx, st.gamma, dt, integ, recon, "roe")
            t += dt
        return np.abs(U[1:4] / U[0]).mean()
    v16, v32 = vmean(16), vmean(32)
    assert v32 < 2e-3
    assert v16 / v32 > 3.3


# --- Toro's exact Riemann solver for the Euler equations (ch. 4) ------------

def exact_euler(wl, wr, g, xi):
    rl, ul, pl = wl; rr, ur, pr = wr
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)

    def fk(p, rk, pk, ak):
        if p > pk:
            A = 2 / ((g + 1) * rk); Bk = (g - 1) / (g + 1) * pk
            return (p - pk) * math.sqrt(A / (p + Bk))
        return 2 * ak / (g - 1) * ((p / pk) ** ((g - 1) / (2 * g)) - 1)

    lo, hi = 1e-12, 100.0 * max(pl, pr)
    for _ in range(200):
        p = 0.5 * (lo + hi)
        if fk(p, rl, pl, al) + fk(p, rr, pr, ar) + ur - ul > 0:
            hi = p
        else:
            lo = p
    ps = 0.5 * (lo + hi)
    us = 0.5 * (ul + ur) + 0.5 * (fk(ps, rr, pr, ar) - fk(ps, rl, pl, al))
    out = np.zeros((len(xi), 3))
    for m, s in enumerate(xi):
        if s <= us:   # left of the contact
            if ps > pl:
                rs = rl * ((ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1))
                S = ul - al * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                out[m] = (rl, ul, pl) if s < S else (rs, us, ps)
            else:
                rs = rl * (ps / pl) ** (1 / g); asl = al * (ps / pl) ** ((g - 1) / (2 * g))
                if s < ul - al:
                    out[m] = (rl, ul, pl)
                elif s > us - asl:
                    out[m] = (rs, us, ps)
                else:
                    u = 2 / (g + 1) * (al + (g - 1) / 2 * ul + s)
                    c = 2 / (g + 1) * (al + (g - 1) / 2 * (ul - s))
                    r = rl * (c / al) ** (2 / (g - 1))
                    out[m] = (r, u, pl * (c / al) ** (2 * g / (g - 1)))
        else:
            if ps > pr:
                rs = rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1))
                S = ur + ar * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                out[m] = (rr, ur, pr) if s > S else (rs, us, ps)
            else:
                rs = rr * (ps / pr) ** (1 / g); asr = ar * (ps / pr) ** ((g - 1) / (2 * g))
                if s > ur + ar:
                    out[m] = (rr, ur, pr)
                elif s < us + asr:
                    out[m] = (rs, us, ps)
                else:
                    u = 2 / (g + 1) * (-ar + (g - 1) / 2 * ur + s)
                    c = 2 / (g + 1) * (ar - (g - 1) / 2 * (ur - s))
                    r = rr * (c / ar) ** (2 / (g - 1))
                    out[m] = (r, u, pr * (c / ar) ** (2 * g / (g - 1)))
    return out


@pytest.mark.parametrize("integ,recon,solver", COMBOS)
def test_sod_converges_to_exact_euler(integ, recon, solver):
    g = 1.4
    wl, wr = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)

    def err(n):
        dx = 1.0 / n
        x = (np.arange(n) + 0.5) * dx
        left = (x >= 0.25) & (x < 0.75)    # two Riemann problems on the periodic line
        rho = np.where(left, wl[0], wr[0]); P = np.where(left, wl[2], wr[2])
        z = np.zeros(n)
        Bf = np.zeros((3, 1, 1, n))
        U = I.conserved(rho[None, None], z[None, None], z[None, None], z[None, None], P[None, None], Bf, g)
        B = np.ascontiguousarray(Bf)
        t, T = 0.0, 0.1
        while t < T:
            dt = min(orc.cfl_dt(U, B, dx, g, 0.4), T - t)
            orc.step(U, B, dx, g, dt, integ, recon, solver)
            t += dt
        # compare around the discontinuity at x = 0.75 (L state on its left)
        sel = (x > 0.5) & (x < 1.0)
        ex = exact_euler(wl, wr, g, (x[sel] - 0.75) / T)
        return np.abs(U[0, 0, 0, sel] - ex[:, 0]).mean()

    e128, e512 = err(128), err(512)
    assert e512 < 4e-3
    assert e128 / e512 > 2.2          # at least ~first order across discontinuities


def test_cfl_closed_forms():
    g = 5.0 / 3.0
    st = I.uniform(4, rho=2.0, v=(0.3, -0.1, 0.05), P=1.2, Bv=(0.0, 0.0, 0.0), gamma=g)
    a = math.sqrt(g * 1.2 / 2.0)
    assert math.isclose(orc.cfl_dt(st.U, st.B, st.dx, g, 0.3), 0.3 * st.dx / (0.3 + a), rel_tol=1e-14)
    st = I.uniform(4, rho=2.0, v=(0.0, 0.0, 0.0), P=1.2, Bv=(1.5, 0.0, 0.0), gamma=g)
    ca = 1.5 / math.sqrt(2.0)
    smax = max(max(a, ca), math.sqrt(a * a + ca * ca))
    assert math.isclose(orc.cfl_dt(st.U, st.B, st.dx, g, 0.3), 0.3 * st.dx / smax, rel_tol=1e-14)


def test_pressure_floor_raises_energy_only():
    """The optional pressure floor (used for the blast and low-beta stress
    states; not part of the paper's scheme): with pfloor = 0 the floored step
    is the plain step bit for bit; with a floor, exactly the cells whose P is
    below it at the start of the step are counted, and the step conserves
    mass, momentum and face B as before while the energy sum grows by the
    raise sum_c (pfloor - P_c)/(gamma - 1)."""
    st = I.abc(16, kmult=1, beta=1.0, seed=3)
    U, B = st.U.copy(), st.B.copy()
    W0 = orc.prim(U, B, st.gamma)
    # lower the energy of a few cells so that their pressure is below the floor
    cells = [(1, 2, 3), (7, 7, 7), (15, 0, 9), (4, 11, 2)]
    for (k, j, i) in cells:
        U[4, k, j, i] -= (W0[4, k, j, i] + 0.05) / (st.gamma - 1.0)
    pf = 0.02
    W1 = orc.prim(U, B, st.gamma)
    low = W1[4] < pf
    assert int(low.sum()) == len(cells)
    raise_sum = float(((pf - W1[4][low]) / (st.gamma - 1.0)).sum())
    dt = orc.cfl_dt(U, B, st.dx, st.gamma, 0.3, pfloor=pf)
    assert dt > 0 and math.isfinite(dt)
    Ua, Ba = U.copy(), B.copy()
    Ub, Bb = U.copy(), B.copy()
    orc.step(Ua, Ba, st.dx, st.gamma, dt, "vl", "plm", "hlld")
    fb, nf = orc.step_floor(Ub, Bb, st.dx, st.gamma, dt, "vl", "plm", "hlld", pfloor=0.0)
    assert nf == 0 and np.array_equal(Ua, Ub) and np.array_equal(Ba, Bb)
    s0 = orc.sums(U, B)
    Uc, Bc = U.copy(), B.copy()
    fb, nf = orc.step_floor(Uc, Bc, st.dx, st.gamma, dt, "vl", "plm", "hlld", pfloor=pf)
    assert nf == len(cells)
    s1 = orc.sums(Uc, Bc)
    scale = np.abs(U).reshape(5, -1).sum(axis=1)
    for f in (0, 1, 2, 3):
        assert abs(s1[f] - s0[f]) <= 1e-13 * scale[f] + 1e-13
    assert abs(s1[4] - (s0[4] + raise_sum)) <= 1e-12 * scale[4]
    for d in range(3):
        assert abs(s1[5 + d] - s0[5 + d]) <= 1e-13 * np.abs(B[d]).sum()
