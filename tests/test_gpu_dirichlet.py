"""Dirichlet sides on the GPU (mhd_set_dirichlet: fixed-state ghost layers
inside the box, put back after every step) against the oracle's: FP64
parity at the 1e-12 bar along every axis and for each reconstruction and
solver, VL and CTU; the interior independent of the layer count beyond the
minimum (the GPU with the fewest layers against the oracle with six); the
Table 1 RJ2a tube of the paper's setup (box length 1, CTU, PPM, Roe, FP64)
advanced on the GPU alone; the FP32 form's L1 against the FP64 oracle; the
refusals."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1804_03479_b300 import inputs as I

pytestmark = pytest.mark.gpu

GAM = 5.0 / 3.0
GOLDEN = __file__.replace("test_gpu_dirichlet.py", "golden/table1_riemann_states.txt")
# no velocity component vanishes identically: the edge-field upwinding takes
# the side of the sign of the face mass flux, and a flux that is zero in
# exact arithmetic but not after the characteristic projection (round-off
# either side of zero) can be taken differently by two correct programs
W_IN = np.array([1.0, 1.5, 0.1, -0.08, 1.0, 0.7, 0.6, 0.2])
W_BOX = np.array([0.5, 0.2, 0.05, 0.07, 0.4, 0.7, 0.3, -0.1])


@pytest.fixture(scope="module")
def M():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_03479_b300 import mhd
    mhd.lib()
    return mhd


def rel_l1(a, b):
    den = np.abs(b).sum()
    return np.abs(a - b).sum() / (den if den > 0 else 1.0)


def x_problem(n, nl, w_in, w_box, m=(6, 5), seed=3):
    """interior of n cells along x holding w_box with 3-D transverse-velocity
    noise near the lower end, nl ghost layers each end (lower: w_in, upper:
    w_box); m = (cells along y, cells along z)"""
    dx = 1.0 / n
    N = n + 2 * nl
    x = (np.arange(N) - nl + 0.5) * dx
    shp = (m[1], m[0], N)
    f = [np.broadcast_to(np.where(x < 0.0, a, b), shp).copy() for a, b in zip(w_in, w_box)]
    pad = np.zeros(shp)
    pad[:, :, nl:nl + n] = np.random.default_rng(seed).uniform(-1.0, 1.0, (m[1], m[0], n))
    f[2] = f[2] + 0.05 * pad * (np.abs(x - 0.15) < 0.15)
    Bf = np.stack(f[5:8])
    return I.conserved(f[0], f[1], f[2], f[3], f[4], Bf, GAM), np.ascontiguousarray(Bf), dx


def relabel(U, B, w_lo, w_hi, times):
    """carry a problem along x to axis `times` by the cyclic relabelling
    x -> y -> z (array axes, vector components and the Dirichlet states)"""
    for _ in range(times):
        U = np.ascontiguousarray(np.stack([U[0], U[3], U[1], U[2], U[4]]).transpose(0, 2, 3, 1))
        B = np.ascontiguousarray(np.stack([B[2], B[0], B[1]]).transpose(0, 2, 3, 1))
        w_lo = w_lo[[0, 3, 1, 2, 4, 7, 5, 6]]
        w_hi = w_hi[[0, 3, 1, 2, 4, 7, 5, 6]]
    return U, B, w_lo, w_hi


def parity(M, U, B, dx, scheme, axis, nl, w_lo, w_hi, nsteps, sweeps=None, tol=1e-12):
    U, B = U.copy(), B.copy()
    orc.fix_layers(U, B, GAM, axis, nl, w_lo, w_hi)
    s = M.Solver(U.shape[1:], dx, GAM, *scheme, "fp64", 0.3)
    try:
        s.set_dirichlet(axis, nl, w_lo, w_hi)
        assert s.dirichlet(axis) == nl and s.boundary() == 1 << axis
        if sweeps is not None:
            s.set_sweep_pencils(*sweeps)
        for it in range(nsteps):
            s.set_state(U, B)
            dt = orc.cfl_dt(U, B, dx, GAM, 0.3, bc=1 << axis)
            assert abs(s.cfl_dt() - dt) <= 1e-14 * dt
            s.step(dt)
            orc.step_dirichlet(U, B, dx, GAM, dt, *scheme, axis, nl, w_lo, w_hi)
            Ug, Bg = s.get_state()
            for f in range(5):
                assert rel_l1(Ug[f], U[f]) <= tol, (scheme, axis, it, f, rel_l1(Ug[f], U[f]))
            for d in range(3):
                assert rel_l1(Bg[d], B[d]) <= tol, (scheme, axis, it, d)
    finally:
        s.free()


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("scheme,nl", [(("vl", "plm", "roe"), 2), (("vl", "ppm", "hlld"), 3),
                                       (("vl", "plm_prim", "hlle"), 2), (("vl", "ppm", "roe"), 4),
                                       (("ctu", "ppm", "roe"), 2), (("ctu", "plm", "hlld"), 3)])
def test_dirichlet_fp64_parity(M, axis, scheme, nl):
    U, B, dx = x_problem(40, nl, W_IN, W_BOX)
    U, B, lo, hi = relabel(U, B, W_IN, W_BOX, axis)
    parity(M, U, B, dx, scheme, axis, nl, lo, hi, 4)


@pytest.mark.parametrize("sweeps", [(0, 16), (6, 8)])
def test_dirichlet_fp64_parity_sweep_forms(M, sweeps):
    U, B, dx = x_problem(48, 3, W_IN, W_BOX, m=(20, 9))
    parity(M, U, B, dx, ("vl", "ppm", "roe"), 0, 3, W_IN, W_BOX, 3, sweeps=sweeps)


@pytest.mark.parametrize("scheme,nl", [(("vl", "plm", "roe"), 2), (("vl", "ppm", "hlld"), 3),
                                       (("ctu", "ppm", "roe"), 2)])
def test_fewest_layers_match_six(M, scheme, nl):
    """the GPU with the minimum layer count, advanced on its own (its own
    CFL dt, device graph), against the oracle with six layers: the interior
    agrees at the parity bar"""
    n, steps = 40, 6
    Ug0, Bg0, dx = x_problem(n, nl, W_IN, W_BOX)
    Uo, Bo, _ = x_problem(n, 6, W_IN, W_BOX)
    orc.fix_layers(Uo, Bo, GAM, 0, 6, W_IN, W_BOX)
    s = M.Solver(Ug0.shape[1:], dx, GAM, *scheme, "fp64", 0.3)
    try:
        s.set_dirichlet(0, nl, W_IN, W_BOX)
        s.set_state(Ug0, Bg0)
        s.advance(steps)
        Ug, Bg = s.get_state()
    finally:
        s.free()
    for _ in range(steps):
        dt = orc.cfl_dt(Uo, Bo, dx, GAM, 0.3, bc=1)
        orc.step_dirichlet(Uo, Bo, dx, GAM, dt, *scheme, 0, 6, W_IN, W_BOX)
    for f in range(5):
        assert rel_l1(Ug[f][..., nl:nl + n], Uo[f][..., 6:6 + n]) <= 1e-12, f
    for d in range(3):
        assert rel_l1(Bg[d][..., nl:nl + n + 1], Bo[d][..., 6:6 + n + 1]) <= 1e-12, d


def rj2a_line(n, nl):
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        tok = line.split()
        rows[tok[0]] = [float(eval(t, {"math": math})) for t in tok[1:]]
    v = rows["rj2a"]
    wl = np.array([v[0], v[1], v[2], v[3], v[4], v[14], v[5], v[6]])
    wr = np.array([v[7], v[8], v[9], v[10], v[11], v[14], v[12], v[13]])
    dx = 1.0 / n
    x = (np.arange(n + 2 * nl) - nl + 0.5) * dx
    shp = (2, 2, n + 2 * nl)
    f = [np.broadcast_to(np.where(x < 0.5, a, b), shp).copy() for a, b in zip(wl, wr)]
    Bf = np.stack(f[5:8])
    return I.conserved(f[0], f[1], f[2], f[3], f[4], Bf, GAM), np.ascontiguousarray(Bf), dx, wl, wr


@pytest.mark.parametrize("integ", ["ctu", "vl"])
def test_rj2a_paper_setup_on_the_gpu(M, integ):
    """RJ2a (Table 1) in a box of length 1 with Dirichlet ends, PPM + Roe in
    FP64 (the paper's accuracy tests use CTU), advanced by the GPU alone to
    t = 0.2 (the fast waves reach the ends at about t = 0.2): against the
    oracle's run at every 40th step, and the end states kept in the ghost
    layers"""
    n, nl = 192, 3
    U, B, dx, wl, wr = rj2a_line(n, nl)
    Uo, Bo = U.copy(), B.copy()
    orc.fix_layers(Uo, Bo, GAM, 0, nl, wl, wr)
    s = M.Solver(U.shape[1:], dx, GAM, integ, "ppm", "roe", "fp64", 0.3)
    try:
        s.set_dirichlet(0, nl, wl, wr)
        s.set_state(U, B)
        t, it = 0.0, 0
        while t < 0.2:
            dt = min(s.cfl_dt(), 0.2 - t)
            do = orc.cfl_dt(Uo, Bo, dx, GAM, 0.3, bc=1)
            assert abs(min(do, 0.2 - t) - dt) <= 1e-12 * dt
            s.step(dt)
            orc.step_dirichlet(Uo, Bo, dx, GAM, dt, integ, "ppm", "roe", 0, nl, wl, wr)
            t += dt
            it += 1
            if it % 40 == 0:
                Ug, _ = s.get_state()
                for f in range(5):
                    assert rel_l1(Ug[f], Uo[f]) <= 1e-11, (it, f)
        Ug, Bg = s.get_state()
    finally:
        s.free()
    for f in range(5):
        assert rel_l1(Ug[f], Uo[f]) <= 1e-11, f
    W = orc.prim(Ug, Bg, GAM, bc=1)
    assert W[0].min() > 0 and W[4].min() > 0
    assert np.allclose(W[0, :, :, :nl], wl[0], rtol=1e-14) and np.allclose(W[0, :, :, -nl:], wr[0], rtol=1e-14)
    assert np.abs(Bg[0] - wl[5]).max() <= 1e-13            # the normal field stays uniform


def test_dirichlet_fp32_against_fp64_oracle(M):
    """FP32 form: per-field relative L1 against the FP64 oracle after 10 steps"""
    U, B, dx = x_problem(48, 3, W_IN, W_BOX)
    Uo, Bo = U.copy(), B.copy()
    orc.fix_layers(Uo, Bo, GAM, 0, 3, W_IN, W_BOX)
    s = M.Solver(U.shape[1:], dx, GAM, "vl", "ppm", "hlld", "fp32", 0.3)
    try:
        s.set_dirichlet(0, 3, W_IN, W_BOX)
        s.set_state(U.astype(np.float32), B.astype(np.float32))
        for _ in range(10):
            dt = orc.cfl_dt(Uo, Bo, dx, GAM, 0.3, bc=1)
            s.step(dt)
            orc.step_dirichlet(Uo, Bo, dx, GAM, dt, "vl", "ppm", "hlld", 0, 3, W_IN, W_BOX)
        Ug, Bg = s.get_state()
    finally:
        s.free()
    for f in range(5):
        assert rel_l1(Ug[f].astype(np.float64), Uo[f]) <= 2e-5, f
    for d in range(3):
        assert rel_l1(Bg[d].astype(np.float64), Bo[d]) <= 2e-5, d


def test_dirichlet_refusals(M):
    U, B, dx = x_problem(16, 3, W_IN, W_BOX, m=(4, 4))
    s = M.Solver(U.shape[1:], dx, GAM, "vl", "ppm", "roe", "fp64", 0.3)
    try:
        for args in [(3, 3, W_IN, W_BOX), (0, 2, W_IN, W_BOX), (0, 11, W_IN, W_BOX),
                     (0, 3, np.array([-1.0, 0, 0, 0, 1, 0, 0, 0]), W_BOX),
                     (0, 3, W_IN, np.array([1.0, 0, 0, 0, 0.0, 0, 0, 0])),
                     (0, 3, W_IN, np.array([1.0, 0, 0, 0, np.nan, 0, 0, 0]))]:
            with pytest.raises(RuntimeError):
                s.set_dirichlet(*args)
            s.clear_error()
        s.set_dirichlet(0, 3, W_IN, W_BOX)
        assert s.dirichlet(0) == 3 and s.boundary() == 1
        s.set_dirichlet(0, 0)
        assert s.dirichlet(0) == 0 and s.boundary() == 1
        s.set_dirichlet(0, 3, W_IN, W_BOX)
        s.set_boundary(0)
        assert s.dirichlet(0) == 0 and s.boundary() == 0
    finally:
        s.free()
    # CTU needs two layers whatever the reconstruction; batches are refused
    s = M.Solver(U.shape[1:], dx, GAM, "ctu", "ppm", "roe", "fp64", 0.3)
    try:
        s.set_dirichlet(0, 2, W_IN, W_BOX)
        assert s.dirichlet(0) == 2
        with pytest.raises(RuntimeError):
            s.set_dirichlet(0, 1, W_IN, W_BOX)
    finally:
        s.free()
    s = M.Solver(None, None, GAM, "vl", "plm", "roe", "fp64", 0.3, shapes=[(16, 8, 8), (16, 8, 8)], dxs=[0.1, 0.1])
    try:
        with pytest.raises(RuntimeError):
            s.set_dirichlet(0, 2, W_IN, W_BOX)
    finally:
        s.free()
