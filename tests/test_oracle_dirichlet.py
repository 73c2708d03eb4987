"""Dirichlet sides of the oracle (the shock tubes of Sec. 5.1 hold the left
and right states at the two ends of the box): nl ghost layers inside the box
kept at a fixed state and put back after every step, with the outflow rule
beyond them.  Pinned by: supersonic inflow through a Dirichlet side against
the same inflow from a wide upstream region of the fixed state on a periodic
line (no boundary at all); a box fed by a supersonic stream through both
sides relaxing to that stream; the minimum layer counts (2 for PLM, 3 for
PPM), beyond which more layers change nothing; and the Table 1 RJ2a tube,
whose result equals the outflow one until its waves reach the ends.  Both
integrators, VL and CTU (the paper's accuracy tests use CTU)."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1804_03479_b300 import inputs as I

GAM = 5.0 / 3.0
GOLDEN = __file__.replace("test_oracle_dirichlet.py", "golden/table1_riemann_states.txt")


def line_state(prof, n, m=2, seed=None, noise_region=None, x=None):
    """(U, B) of a line along x: prof(x) -> (rho, vx, vy, vz, P, Bx, By, Bz)
    arrays over the n cells; seeded transverse-velocity noise on the cells of
    noise_region (drawn per interior cell so that it does not depend on the
    box padding)"""
    shp = (m, m, n)
    w = [np.broadcast_to(np.asarray(q, float), (n,)) for q in prof]
    f = [np.broadcast_to(q, shp).copy() for q in w]
    if seed is not None:
        rng = np.random.default_rng(seed)
        f[2] = f[2] + 0.02 * rng.uniform(-1.0, 1.0, shp) * noise_region
    Bf = np.stack(f[5:8])
    return I.conserved(f[0], f[1], f[2], f[3], f[4], Bf, GAM), np.ascontiguousarray(Bf)


def interior_noise(n, N, nl, seed, one_d):
    pad = np.zeros((2, 2, N))
    rng = np.random.default_rng(seed)
    pad[:, :, nl:nl + n] = rng.uniform(-1.0, 1.0, n) if one_d else rng.uniform(-1.0, 1.0, (2, 2, n))
    return pad


def boundary_problem(n, nl, w_in, w_box, seed=3, one_d=False):
    """interior of n cells on [0, 1] holding w_box (with transverse-velocity
    noise near the left end, varying along x only if one_d), nl ghost layers
    each side: the left ones hold w_in, the right ones w_box"""
    dx = 1.0 / n
    N = n + 2 * nl
    x = (np.arange(N) - nl + 0.5) * dx
    prof = [np.where(x < 0.0, a, b) for a, b in zip(w_in, w_box)]
    U, B = line_state(prof, N)
    U[2] += 0.02 * interior_noise(n, N, nl, seed, one_d) * U[0] * (np.abs(x - 0.15) < 0.15)
    return U, B, dx


def run_dirichlet(U, B, dx, nl, w_lo, w_hi, steps, scheme, cfl=0.3):
    orc.fix_layers(U, B, GAM, 0, nl, w_lo, w_hi)
    for _ in range(steps):
        dt = orc.cfl_dt(U, B, dx, GAM, cfl, bc=1)
        orc.step_dirichlet(U, B, dx, GAM, dt, *scheme, 0, nl, w_lo, w_hi)
    return U, B


W_IN = np.array([1.0, 1.5, 0.1, 0.0, 1.0, 0.7, 0.6, 0.2])       # subsonic inflow (c_f ~ 1.6)
W_BOX = np.array([0.5, 0.2, 0.0, 0.0, 0.4, 0.7, 0.3, -0.1])


@pytest.mark.parametrize("integ,recon,nmin", [("vl", "plm", 2), ("vl", "plm_prim", 2), ("vl", "ppm", 3),
                                              ("ctu", "plm", 2), ("ctu", "ppm", 2)])
def test_layers_beyond_the_minimum_change_nothing(integ, recon, nmin):
    """the interior after six steps, with a Riemann problem at the left side,
    is the same bit for bit for nmin and 6 layers; with nmin - 1 it is not.
    The first ghost cell's upper face is an interior face, so its cell-centre
    field already differs from the fixed state at the start of a step.  In a
    VL step PPM's interface value at the half step reaches one cell further
    than the PLM slope; CTU reconstructs once, at t^n, so two layers serve
    both."""
    out = {}
    for nl in (nmin - 1, nmin, 6):
        U, B, dx = boundary_problem(48, nl, W_IN, W_BOX)
        U, B = run_dirichlet(U, B, dx, nl, W_IN, W_BOX, 6, (integ, recon, "roe"))
        out[nl] = (U[..., nl:nl + 48], B[..., nl:nl + 49])
    assert np.array_equal(out[nmin][0], out[6][0]) and np.array_equal(out[nmin][1], out[6][1])
    assert np.abs(out[nmin - 1][0] - out[6][0]).max() > 1e-10


@pytest.mark.parametrize("scheme", [("vl", "plm", "roe"), ("vl", "ppm", "hlld"), ("vl", "plm_prim", "hlle"),
                                    ("ctu", "ppm", "roe"), ("ctu", "plm", "hlld")])
def test_supersonic_inflow_equals_a_wide_upstream_region(scheme):
    """every wave of the problem at the left side moves into the box, so the
    interior of this 1-D problem cannot tell the Dirichlet side from a wide
    region of the fixed state upstream (a periodic line, no boundary): the
    two agree to round-off while the wrap of the periodic line is still far
    away.  (With variation across the line the cell-centre field of the
    first upstream cell takes in its upper face, which CT advances, so the
    upstream cells of the periodic line move while the ghost cells are put
    back: the comparison holds for 1-D problems only.)"""
    w_in = np.array([1.0, 3.0, 0.1, 0.0, 0.6, 0.5, 0.3, 0.1])      # v_x = 3 > c_f
    w_box = np.array([0.7, 2.8, 0.0, 0.0, 0.5, 0.5, 0.1, -0.1])    # also supersonic along +x
    n, nl, up, steps = 48, 3, 40, 8
    U, B, dx = boundary_problem(n, nl, w_in, w_box, one_d=True)
    orc.fix_layers(U, B, GAM, 0, nl, w_in, w_box)
    dts = []
    for _ in range(steps):
        dts.append(orc.cfl_dt(U, B, dx, GAM, 0.3, bc=1))
        orc.step_dirichlet(U, B, dx, GAM, dts[-1], *scheme, 0, nl, w_in, w_box)
    # periodic line: `up` cells of w_in, the interior with the same noise, `up` cells of w_box
    N = up + n + up
    x = (np.arange(N) - up + 0.5) * dx
    prof = [np.where(x < 0.0, a, b) for a, b in zip(w_in, w_box)]
    Up, Bp = line_state(prof, N)
    Up[2] += 0.02 * interior_noise(n, N, up, 3, True) * Up[0] * (np.abs(x - 0.15) < 0.15)
    for dt in dts:
        # the bounded run's dt (the wrap of the periodic line, far upstream,
        # makes faster states of its own)
        orc.step(Up, Bp, dx, GAM, dt, *scheme)
    a, b = U[..., nl:nl + n], Up[..., up:up + n]
    for f in range(5):
        assert np.abs(a[f] - b[f]).sum() <= 1e-12 * np.abs(b[f]).sum(), f
    assert np.abs(B[..., nl:nl + n] - Bp[..., up:up + n]).max() <= 1e-12


def test_box_relaxes_to_a_supersonic_stream():
    """a stream entering at the left and held at the right side too flushes
    a box of a different state: after the box has been crossed several
    times every cell holds the stream"""
    w = np.array([1.0, 2.5, 0.0, 0.0, 0.5, 0.4, 0.2, 0.0])
    n, nl = 32, 3
    U, B, dx = boundary_problem(n, nl, w, np.array([0.4, 0.0, 0.0, 0.0, 0.2, 0.4, -0.3, 0.1]))
    orc.fix_layers(U, B, GAM, 0, nl, w, w)
    t, dev = 0.0, []
    for t_end in (2.0, 6.0):
        while t < t_end:
            dt = orc.cfl_dt(U, B, dx, GAM, 0.4, bc=1)
            orc.step_dirichlet(U, B, dx, GAM, dt, "vl", "plm", "hlld", 0, nl, w, w)
            t += dt
        W = orc.prim(U, B, GAM, bc=1)
        dev.append(max(np.abs(W[f] - w[f]).max() for f in range(5)))
    assert dev[1] <= 1e-7 and dev[1] < 0.1 * dev[0], dev      # from O(1) at t = 0
    assert np.abs(B[1] - w[6]).max() <= 1e-7 and np.abs(B[0] - w[5]).max() <= 1e-7


@pytest.mark.parametrize("integ", ["ctu", "vl"])
def test_rj2a_tube_equals_the_outflow_tube_until_its_waves_arrive(integ):
    """Table 1 RJ2a with Dirichlet sides (the paper's setup: box length 1,
    CTU, PPM, Roe, FP64): while its fastest waves are inside the box the
    ghost layers stay at the end states, so the result is the outflow one"""
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        tok = line.split()
        rows[tok[0]] = [float(eval(t, {"math": math})) for t in tok[1:]]
    v = rows["rj2a"]
    wl = np.array([v[0], v[1], v[2], v[3], v[4], v[14], v[5], v[6]])
    wr = np.array([v[7], v[8], v[9], v[10], v[11], v[14], v[12], v[13]])
    n, nl = 128, 3
    dx = 1.0 / n
    x = (np.arange(n + 2 * nl) - nl + 0.5) * dx
    U, B = line_state([np.where(x < 0.5, a, b) for a, b in zip(wl, wr)], n + 2 * nl, m=1)
    Uo, Bo = U.copy(), B.copy()
    orc.fix_layers(U, B, GAM, 0, nl, wl, wr)
    # the layers already held the end states (up to the rounding of e)
    assert np.abs(U - Uo).max() <= 1e-15 * np.abs(Uo).max() and np.array_equal(B, Bo)
    t = 0.0
    while t < 0.1:            # fast waves of RJ2a travel below 2.4: they stay inside [0, 1]
        dt = orc.cfl_dt(U, B, dx, GAM, 0.3, bc=1)
        orc.step_dirichlet(U, B, dx, GAM, dt, integ, "ppm", "roe", 0, nl, wl, wr)
        orc.step_bc(Uo, Bo, dx, GAM, dt, integ, "ppm", "roe", bc=1)
        t += dt
    # to round-off: the uniform end regions of the outflow run pick up an
    # ulp here and there, the ghost layers of the Dirichlet run are rewritten
    assert np.abs(U[..., nl:nl + n] - Uo[..., nl:nl + n]).max() <= 1e-13
    assert np.abs(B[..., nl:nl + n + 1] - Bo[..., nl:nl + n + 1]).max() <= 1e-13
    W = orc.prim(U, B, GAM, bc=1)
    assert W[0].min() > 0 and W[4].min() > 0
    # the waves did move: the middle differs from both end states
    assert np.abs(W[0, 0, 0, n // 2 - 20:n // 2 + 20] - wl[0]).max() > 0.05


def test_fix_layers_keeps_the_interior_upper_face():
    U, B = line_state([np.ones(10)] * 8, 10, m=1)
    B[0] = np.arange(10.0)
    w = np.array([1.0, 0.0, 0.0, 0.0, 1.0, -5.0, 0.0, 0.0])
    orc.fix_layers(U, B, GAM, 0, 2, w, w)
    assert list(B[0, 0, 0]) == [-5, -5, 2, 3, 4, 5, 6, 7, 8, -5]
