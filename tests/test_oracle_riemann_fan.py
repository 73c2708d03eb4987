"""Riemann fans of the oracle's solvers (Sec. 3.2: Roe, HLLD, HLLE) checked
against what the mathematics and brute force fix.

Fan structure (the oracle exports each solver's fan: orc_hlld_fan,
orc_hlle_fan, orc_roe_waves):
- HLLD (Miyoshi & Kusano 2005): S_L < S_M < S_R always; S*_L <= S_M <= S*_R
  by construction; S_L <= S*_L holds exactly when the left single-star
  denominator rho_L (u_L - S_L)(S_M - S_L) - B_n^2 is >= 0 (and likewise on
  the right), which the method's speed estimate min(u) - max(c_f) does not
  guarantee for every pair of states: the full ordering
  S_L <= S*_L <= S_M <= S*_R <= S_R holds on the Table 1 problems and on all
  but about one in 2000 random pairs;
- the integral of each fan equals the HLL average: the sum over the fan of
  (width x state) is S_R U_R - S_L U_L - (F_R - F_L) (the integral form of
  the conservation law over [S_L t, S_R t]); the flux is F_L plus the jumps
  of the waves with negative speed (Rankine-Hugoniot across each wave);
- Roe: the seven eigenvalues of the linearisation are ordered and the flux
  is F_L + sum over negative eigenvalues of lambda eta r.

Brute force (a finely resolved 1-D run, 2^14 cells, of the oracle's own VL
step with the same solver, sampled at x/t = 0):
- isolated moving discontinuities a solver resolves exactly (a contact for
  Roe and HLLD, a perpendicular fast shock from the jump conditions for
  Roe): the run's state at x/t = 0 is the upwind state and the solver's
  one-step flux is its physical flux, to round-off (a moving rotational
  discontinuity is checked for exactness without a run);
- the Table 1 problems (Sec. 5.1 (ii)), Galilean-boosted so that x/t = 0
  lies mid-way between two of the Roe eigenvalues: outside [S_L t, S_R t]
  (HLLE and HLLD speed bounds, 12 cells of numerical precursor allowed) the
  run is still the initial state; its integral over the fan is the HLL
  average; the three solvers' runs reach the same state at x/t = 0; and
  each solver's one-step flux lies within a stated fraction of the jump
  |F_R - F_L| of the brute-force Godunov flux F(W(x/t = 0)).  Measured
  fractions (Torrilhon, RJ2a): HLLD 0.23, 0.05; Roe 0.18, 0.02; HLLE 0.65,
  0.03 -- HLLE merges the inner waves, which costs most in Torrilhon's fan.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1804_03479_b300 import inputs as I
from test_oracle_riemann import GAMMA, cons, flux_eq7, random_pairs, table1

N_FINE = 1 << 14


# ---------------------------------------------------------------- fan shape

def test_hlld_fan_ordering_table1():
    for name, wl, wr, bx in table1():
        S, _ = orc.hlld_fan(wl, wr, bx, GAMMA)
        assert np.all(np.diff(S) >= 0.0), (name, S)
        assert S[0] < S[2] < S[4], name


def moderate_pairs(n, seed):
    """jumps within a factor of two, velocities below the sound speed"""
    rng = np.random.default_rng(seed)
    for _ in range(n):
        w = np.array([rng.uniform(0.5, 2), *rng.uniform(-0.5, 0.5, 3), rng.uniform(0.5, 2),
                      *rng.uniform(-1, 1, 2)])
        w2 = w * np.array([rng.uniform(0.5, 2), 1, 1, 1, rng.uniform(0.5, 2), 1, 1])
        w2[[1, 2, 3, 5, 6]] += rng.uniform(-0.5, 0.5, 5)
        yield w, w2, rng.uniform(-1.5, 1.5)


def test_hlld_fan_ordering_random():
    nviol = 0
    for wl, wr, bn in random_pairs(4000, 21):
        S, U = orc.hlld_fan(wl, wr, bn, GAMMA)
        assert S[0] < S[2] < S[4]
        assert S[1] <= S[2] <= S[3]
        den_l = wl[0] * (wl[1] - S[0]) * (S[2] - S[0]) - bn * bn
        den_r = wr[0] * (S[4] - wr[1]) * (S[4] - S[2]) - bn * bn
        # S_L <= S*_L exactly when the left denominator is >= 0 (up to rounding)
        tol = 1e-12 * (wl[0] * (wl[1] - S[0]) * (S[2] - S[0]) + bn * bn)
        if abs(den_l) > tol:
            assert (S[0] <= S[1]) == (den_l > 0), (wl, wr, bn, S)
        tol = 1e-12 * (wr[0] * (S[4] - wr[1]) * (S[4] - S[2]) + bn * bn)
        if abs(den_r) > tol:
            assert (S[3] <= S[4]) == (den_r > 0), (wl, wr, bn, S)
        nviol += not (S[0] <= S[1] and S[3] <= S[4])
    # the speed estimate breaks the full ordering only rarely (2 of these
    # 4000 pairs, 1 of 4000 moderate ones), always with a negative denominator
    assert nviol <= 4
    nviol = 0
    for wl, wr, bn in moderate_pairs(4000, 22):
        S, _ = orc.hlld_fan(wl, wr, bn, GAMMA)
        if not np.all(np.diff(S) >= 0.0):
            nviol += 1
            den_l = wl[0] * (wl[1] - S[0]) * (S[2] - S[0]) - bn * bn
            den_r = wr[0] * (S[4] - wr[1]) * (S[4] - S[2]) - bn * bn
            assert min(den_l, den_r) < 0.0
    assert nviol <= 4


def fan_integral_residual(S, states, ul, ur, fl, fr):
    integ = sum((S[k] - S[k - 1]) * states[k] for k in range(1, len(S)))
    want = S[-1] * ur - S[0] * ul - (fr - fl)
    scale = np.abs(S[-1] * ur).max() + np.abs(S[0] * ul).max() + np.abs(fr).max() + np.abs(fl).max()
    return np.abs(integ - want).max() / scale


def flux_from_fan(S, states, fl):
    f = fl.copy()
    for k in range(len(S)):
        if S[k] < 0.0:
            f = f + S[k] * (states[k + 1] - states[k])
    return f


def all_pairs():
    yield from ((wl, wr, bx) for _, wl, wr, bx in table1())
    yield from random_pairs(2000, 23)
    yield from moderate_pairs(2000, 24)


def test_hlld_fan_integral_is_the_hll_average_and_gives_the_flux():
    for wl, wr, bn in all_pairs():
        S, U = orc.hlld_fan(wl, wr, bn, GAMMA)
        ul, ur = cons(wl, bn, GAMMA), cons(wr, bn, GAMMA)
        fl, fr = flux_eq7(wl, bn, GAMMA), flux_eq7(wr, bn, GAMMA)
        assert np.array_equal(U[0], ul) or np.allclose(U[0], ul, rtol=1e-15, atol=1e-15)
        assert fan_integral_residual(S, U, ul, ur, fl, fr) <= 1e-13
        f, _ = orc.riemann("hlld", wl, wr, bn, GAMMA)
        if S[0] < 0.0 < S[4]:
            g = flux_from_fan(S, U, fl)
            assert np.abs(g - f).max() <= 1e-13 * (1.0 + np.abs(fl).max() + np.abs(fr).max())
        # the normal velocity of every star state is S_M (the contact)
        for k in (1, 2, 3, 4):
            assert abs(U[k][1] / U[k][0] - S[2]) <= 1e-12 * (1.0 + abs(S[2]))


def test_hlle_fan_integral_and_flux():
    for wl, wr, bn in all_pairs():
        S, Uh = orc.hlle_fan(wl, wr, bn, GAMMA)
        ul, ur = cons(wl, bn, GAMMA), cons(wr, bn, GAMMA)
        fl, fr = flux_eq7(wl, bn, GAMMA), flux_eq7(wr, bn, GAMMA)
        assert S[0] < S[1]
        assert fan_integral_residual(S, [ul, Uh, ur], ul, ur, fl, fr) <= 1e-13
        f, _ = orc.riemann("hlle", wl, wr, bn, GAMMA)
        g = flux_from_fan(S, [ul, Uh, ur], fl) if S[1] > 0.0 else fr
        assert np.abs(g - f).max() <= 1e-12 * (1.0 + np.abs(fl).max() + np.abs(fr).max())


def test_roe_fan_ordered_and_gives_the_flux():
    for wl, wr, bn in all_pairs():
        ok, lam, eta, ru = orc.roe_waves(wl, wr, bn, GAMMA)
        if not ok:
            continue
        assert np.all(np.diff(lam) >= -1e-14 * (1 + np.abs(lam).max()))
        f, fb = orc.riemann("roe", wl, wr, bn, GAMMA)
        if fb:
            continue          # fell back to HLLE (a fan state not physical)
        fl = flux_eq7(wl, bn, GAMMA)
        g = fl + sum(lam[a] * eta[a] * ru[a] for a in range(7) if lam[a] < 0.0)
        assert np.abs(g - f).max() <= 1e-10 * (1.0 + np.abs(fl).max())


# -------------------------------------------------------------- brute force

def tube_state(wl, wr, bn, n=N_FINE):
    """1-D Riemann problem along x on n cells (interface at the lower face of
    cell n/2), y and z one cell each."""
    shp = (1, 1, n)
    left = np.arange(n) < n // 2

    def col(k):
        return np.where(left, wl[k], wr[k]).reshape(shp).astype(float)
    B = np.stack([np.full(shp, float(bn)), col(5), col(6)])
    U = I.conserved(col(0), col(1), col(2), col(3), col(4), B, GAMMA)
    return U, B


def fine_run(wl, wr, bn, solver, nsteps, cfl=0.8, n=N_FINE):
    """VL + PLM with `solver` and outflow ends; returns U, B and the time."""
    U, B = tube_state(wl, wr, bn, n)
    dx, t = 1.0 / n, 0.0
    for _ in range(nsteps):
        dt = orc.cfl_dt(U, B, dx, GAMMA, cfl, bc=1)
        orc.step_bc(U, B, dx, GAMMA, dt, "vl", "plm", solver, bc=1)
        t += dt
    return U, B, t


def sweep_cons(U, B):
    """conserved sweep-frame rows (rho, Mx, My, Mz, e, By, Bz) along the line"""
    return np.stack([U[0, 0, 0], U[1, 0, 0], U[2, 0, 0], U[3, 0, 0], U[4, 0, 0], B[1, 0, 0], B[2, 0, 0]])


def state_at_zero(U, B, n=N_FINE):
    """primitive sweep-frame state at x/t = 0: mean of the two cells beside
    the interface, and its spread over the eight nearest cells"""
    W = orc.prim(U, B, GAMMA, bc=1)[:, 0, 0, :]
    c = n // 2
    w0 = 0.5 * (W[:, c - 1] + W[:, c])
    spread = np.abs(W[:, c - 4:c + 4] - w0[:, None]).max()
    return np.array([w0[0], w0[1], w0[2], w0[3], w0[4], w0[6], w0[7]]), spread


def moving_contact(u0):
    wl = np.array([1.3, u0, 0.2, -0.1, 0.8, 0.4, -0.6])
    wr = np.array([0.4, u0, 0.2, -0.1, 0.8, 0.4, -0.6])
    return wl, wr, 0.9


def moving_rotational(s0):
    """an Alfven rotational discontinuity moving at s0: v_n = -c_a + s0"""
    rho, P, bn, bt = 1.1, 0.7, 1.2, 0.8
    ca = abs(bn) / math.sqrt(rho)
    btl = bt * np.array([math.cos(0.3), math.sin(0.3)])
    btr = bt * np.array([math.cos(2.1), math.sin(2.1)])
    vt = np.array([0.1, -0.2])
    vtr = vt - np.sign(bn) * (btr - btl) / math.sqrt(rho)
    wl = np.array([rho, -ca + s0, *vt, P, *btl])
    wr = np.array([rho, -ca + s0, *vtr, P, *btr])
    return wl, wr, bn


def perpendicular_shock(s0):
    """a fast shock with B_n = 0 moving at s0, from the jump conditions
    rho u, rho u^2 + P + B^2/2, B u, u (e + P + B^2/2) continuous across it
    (written in the shock frame, then boosted)"""
    from scipy.optimize import brentq
    g = GAMMA
    rho1, P1, B1, u1 = 1.0, 0.6, 0.8, -3.0           # upstream (right), flowing left in the shock frame

    def resid(r):                                     # r = rho2 / rho1, the compression ratio
        u2, B2, rho2 = u1 / r, B1 * r, rho1 * r
        P2 = rho1 * u1 * u1 + P1 + 0.5 * B1 * B1 - rho2 * u2 * u2 - 0.5 * B2 * B2
        h1 = 0.5 * u1 * u1 + g / (g - 1) * P1 / rho1 + B1 * B1 / rho1
        h2 = 0.5 * u2 * u2 + g / (g - 1) * P2 / rho2 + B2 * B2 / rho2
        return h1 - h2
    r = brentq(resid, 1.0001, 3.999)
    u2, B2, rho2 = u1 / r, B1 * r, rho1 * r
    P2 = rho1 * u1 * u1 + P1 + 0.5 * B1 * B1 - rho2 * u2 * u2 - 0.5 * B2 * B2
    wl = np.array([rho2, u2 + s0, 0.0, 0.0, P2, B2, 0.0])    # downstream on the left
    wr = np.array([rho1, u1 + s0, 0.0, 0.0, P1, B1, 0.0])
    return wl, wr, 0.0


# (name, states, exact solvers, tolerance of the fine run's state at x/t = 0):
# a captured shock leaves start-up and post-shock noise of a few 1e-3 behind
# it, which is the scheme's, not the solver's
EXACT = [("contact", moving_contact(0.35), ("roe", "hlld"), 1e-9),
         ("contact-left", moving_contact(-0.35), ("roe", "hlld"), 1e-9),
         ("fast-shock", perpendicular_shock(0.4), ("roe",), 1e-2)]


def one_discontinuity(wl, wr, bn):
    """(speed, upwind state, its flux) of a single discontinuity; asserts
    that F_R - F_L = s (U_R - U_L) for one speed s"""
    fl, fr = flux_eq7(wl, bn, GAMMA), flux_eq7(wr, bn, GAMMA)
    ul, ur = cons(wl, bn, GAMMA), cons(wr, bn, GAMMA)
    k = np.argmax(np.abs(ur - ul))
    s = (fr - fl)[k] / (ur - ul)[k]
    assert np.allclose(fr - fl, s * (ur - ul), atol=1e-12)
    upwind = wl if s > 0 else wr
    return s, upwind, flux_eq7(upwind, bn, GAMMA)


@pytest.mark.parametrize("s0", [0.3, -0.3, 2.0])
def test_moving_rotational_discontinuity_exact(s0):
    """Roe and HLLD resolve an isolated moving Alfven discontinuity exactly.
    (No fine run here: a smeared rotation lowers |B_t| inside the transition,
    and the total-pressure deficit launches compressive waves that do not
    vanish with resolution -- the non-uniqueness Torrilhon's problem of
    Sec. 5.1 (ii) is about.)"""
    wl, wr, bn = moving_rotational(s0)
    s, upwind, f_up = one_discontinuity(wl, wr, bn)
    assert abs(s - s0) <= 1e-12
    for solver in ("roe", "hlld"):
        f, fb = orc.riemann(solver, wl, wr, bn, GAMMA)
        assert fb == 0
        assert np.abs(f - f_up).max() <= 1e-11 * (1.0 + np.abs(f_up).max()), (solver, f - f_up)


@pytest.mark.parametrize("name,case,solvers,tol", EXACT, ids=[e[0] for e in EXACT])
def test_bruteforce_isolated_discontinuities(name, case, solvers, tol):
    wl, wr, bn = case
    s, upwind, f_up = one_discontinuity(wl, wr, bn)
    for solver in solvers:
        U, B, t = fine_run(wl, wr, bn, solver, 300)
        w0, spread = state_at_zero(U, B)
        # the brute-force run leaves the upwind state at x/t = 0
        assert np.abs(w0 - upwind).max() <= tol * (1.0 + np.abs(upwind).max()), (solver, w0, upwind)
        assert spread <= tol * (1.0 + np.abs(upwind).max())
        f, fb = orc.riemann(solver, wl, wr, bn, GAMMA)
        assert fb == 0
        assert np.abs(f - f_up).max() <= 1e-11 * (1.0 + np.abs(f_up).max()), (solver, f - f_up)
    f, _ = orc.riemann("hlle", wl, wr, bn, GAMMA)
    if name.startswith("contact"):
        # the two-wave solver smears a contact (it is not exact there)
        assert np.abs(f - f_up).max() > 1e-4
    else:
        # an isolated fast shock travels at the Roe average's fast speed, one
        # of Einfeldt's bounds, so the HLL state is exact there too
        assert np.abs(f - f_up).max() <= 1e-11 * (1.0 + np.abs(f_up).max())


FLUX_FRACTION = {"hlld": 0.3, "roe": 0.3, "hlle": 0.75}


@pytest.mark.parametrize("name", [t[0] for t in table1()])
def test_bruteforce_table1_fans(name):
    _, wl, wr, bx = next(t for t in table1() if t[0] == name)
    ok, lam, _, _ = orc.roe_waves(wl, wr, bx, GAMMA)
    assert ok
    k = int(np.argmax(np.diff(lam)))
    u0 = -0.5 * (lam[k] + lam[k + 1])       # x/t = 0 mid-way between two waves
    wl, wr = wl.copy(), wr.copy()
    wl[1] += u0
    wr[1] += u0
    ul, ur = cons(wl, bx, GAMMA), cons(wr, bx, GAMMA)
    fl, fr = flux_eq7(wl, bx, GAMMA), flux_eq7(wr, bx, GAMMA)
    dF = np.abs(fr - fl).max()
    Sd, _ = orc.hlld_fan(wl, wr, bx, GAMMA)
    Se, Uhll = orc.hlle_fan(wl, wr, bx, GAMMA)
    n, dx = N_FINE, 1.0 / N_FINE
    w0s = {}
    for solver in ("hlld", "roe", "hlle"):
        U, B, t = fine_run(wl, wr, bx, solver, 600)
        Uc = sweep_cons(U, B)
        scale = np.abs(ul).max() + np.abs(ur).max()
        # (1) nothing has moved outside the fan bounds (12 cells of precursor allowed)
        xi = ((np.arange(n) + 0.5) - n / 2) * dx / t
        m = 12 * dx / t
        for S in (Sd[[0, 4]], Se):
            outl, outr = xi < S[0] - m, xi > S[1] + m
            assert np.abs(Uc[:, outl] - ul[:, None]).max() <= 1e-6 * scale, (solver, S)
            assert np.abs(Uc[:, outr] - ur[:, None]).max() <= 1e-6 * scale, (solver, S)
        # (2) the run's integral over the Einfeldt fan (plus the margins) is the HLL average
        ia = n // 2 + int(math.floor(Se[0] * t / dx)) - 16
        ib = n // 2 + int(math.ceil(Se[1] * t / dx)) + 16
        xa, xb = (ia - n // 2) * dx, (ib - n // 2) * dx
        integ = Uc[:, ia:ib].sum(axis=1) * dx
        want = (Se[1] - Se[0]) * t * Uhll + (Se[0] * t - xa) * ul + (xb - Se[1] * t) * ur
        assert np.abs(integ - want).max() <= 1e-9 * scale * (xb - xa), solver
        # (3) the state the run reaches at x/t = 0, and the Godunov flux there
        w0, spread = state_at_zero(U, B)
        w0s[solver] = w0
        f, _ = orc.riemann(solver, wl, wr, bx, GAMMA)
        fg = flux_eq7(w0, bx, GAMMA)
        assert np.abs(f - fg).max() <= FLUX_FRACTION[solver] * dF, (solver, np.abs(f - fg).max() / dF)
    # (4) the three solvers' runs converge to the same solution
    ref = w0s["hlld"]
    for solver in ("roe", "hlle"):
        assert np.abs(w0s[solver] - ref).max() <= 3e-2 * np.abs(ref).max(), solver
