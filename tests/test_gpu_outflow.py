"""Outflow (zero-gradient) boundaries on the GPU (mhd_set_boundary) against
the oracle's: FP64 parity at the 1e-12 bar for every outflow mask, VL and
CTU, with the register sweeps and with tiles, on ragged boxes and on a shock
tube whose waves leave the box; div B kept; the unsupported combinations
refused."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1804_03479_b300 import inputs as I

pytestmark = pytest.mark.gpu


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


def parity(M, U, B, dx, gam, scheme, bc, nsteps, sweeps=None, tol=1e-12):
    U, B = U.copy(), B.copy()
    s = M.Solver(U.shape[1:], dx, gam, *scheme, "fp64", 0.3)
    try:
        s.set_boundary(bc)
        assert s.boundary() == bc
        if sweeps is not None:
            s.set_sweep_pencils(*sweeps)
        for it in range(nsteps):
            s.set_state(U, B)
            dt = orc.cfl_dt(U, B, dx, gam, 0.3, bc=bc)
            assert abs(s.cfl_dt() - dt) <= 1e-14 * dt
            s.step(dt)
            orc.step_bc(U, B, dx, gam, dt, *scheme, bc=bc)
            Ug, Bg = s.get_state()
            for f in range(5):
                assert rel_l1(Ug[f], U[f]) <= tol, (scheme, bc, it, f)
            for d in range(3):
                assert rel_l1(Bg[d], B[d]) <= tol, (scheme, bc, it, d)
        m, brms = s.divB()
        mo, _ = orc.divB(B, bc=bc)
        assert m <= 1e-12 * brms + mo
    finally:
        s.free()


@pytest.mark.parametrize("bc", [1, 2, 4, 7, 5])
@pytest.mark.parametrize("scheme", [("vl", "plm", "roe"), ("vl", "ppm", "hlld"), ("vl", "plm_prim", "hlle"),
                                    ("ctu", "plm", "roe"), ("ctu", "ppm", "hlld"), ("ctu", "ppm", "roe")])
def test_outflow_fp64_parity_ragged(M, bc, scheme):
    st = I.open_box((24, 20, 18), seed=11)
    parity(M, st.U, st.B, st.dx, st.gamma, scheme, bc, 3)


@pytest.mark.parametrize("sweeps", [(0, 16), (7, 5), (6, 32)])
def test_outflow_fp64_parity_sweep_forms(M, sweeps):
    st = I.open_box((40, 24, 20), seed=12)
    parity(M, st.U, st.B, st.dx, st.gamma, ("vl", "ppm", "roe"), 7, 3, sweeps=sweeps)


@pytest.mark.parametrize("bc,sweeps", [(6, (7, 16)), (2, (7, 32)), (7, (7, 16)), (5, (1, 8))])
@pytest.mark.parametrize("scheme", [("ctu", "plm", "roe"), ("ctu", "ppm", "hlld")])
def test_outflow_fp64_parity_ctu_sweep_forms(M, bc, sweeps, scheme):
    """CTU with the x bit in the pencil mask: tracing by warps along x where
    x is periodic (bc 6, 2), by tiles where it is an outflow axis (bc 7, 5);
    several warp segments per row (nx = 64)"""
    st = I.open_box((64, 20, 18), seed=13)
    parity(M, st.U, st.B, st.dx, st.gamma, scheme, bc, 3, sweeps=sweeps)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_outflow_tube_waves_leave(M, axis):
    """an MHD Riemann problem (Table 1, RJ2a) centred in a 160-cell line with
    outflow at both ends: advanced by the oracle until its fast waves have
    left, then compared step by step"""
    path = __file__.replace("test_gpu_outflow.py", "golden/table1_riemann_states.txt")
    import math
    for line in open(path):
        if line.startswith("rj2a "):
            v = [float(eval(t, {"math": math})) for t in line.split()[1:]]
    wl, wr, bn = np.array(v[0:7]), np.array(v[7:14]), v[14]
    st = I.shock_tube(wl, wr, bn, 160, axis=axis, m=2, L=1.0)
    # one problem, centred: left state below the middle, right state above
    n = 160
    x = (np.arange(n) + 0.5) / n
    left = x < 0.5
    prof = np.where(left[None, :], wl[:, None], wr[:, None])
    shp = [2, 2, 2]
    shp[2 - axis] = n
    bshape = [1, 1, 1]
    bshape[2 - axis] = n
    fld = lambda a: np.broadcast_to(a.reshape(bshape), shp).copy()
    t1, t2 = (axis + 1) % 3, (axis + 2) % 3
    vel = [None] * 3
    vel[axis], vel[t1], vel[t2] = fld(prof[1]), fld(prof[2]), fld(prof[3])
    Bc = [None] * 3
    Bc[axis] = np.full(shp, bn)
    Bc[t1], Bc[t2] = fld(prof[5]), fld(prof[6])
    Bf = np.ascontiguousarray(np.stack(Bc))
    U = I.conserved(fld(prof[0]), vel[0], vel[1], vel[2], fld(prof[4]), Bf, st.gamma)
    dx = 1.0 / n
    t = 0.0
    while t < 0.25:
        dt = orc.cfl_dt(U, Bf, dx, st.gamma, 0.3, bc=1 << axis)
        orc.step_bc(U, Bf, dx, st.gamma, dt, "vl", "plm", "hlld", bc=1 << axis)
        t += dt
    parity(M, U, Bf, dx, st.gamma, ("vl", "plm", "hlld"), 1 << axis, 4)


def test_outflow_refusals(M):
    st = I.abc(8, kmult=1, beta=1.0)
    s = M.Solver(None, None, 5 / 3, "vl", "plm", "roe", "fp64", 0.3, shapes=[(8, 8, 8), (8, 8, 8)], dxs=[0.1, 0.1])
    try:
        with pytest.raises(M.MHDError):
            s.set_boundary(1)
    finally:
        s.free()
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", "fp64", 0.3)
    try:
        with pytest.raises(M.MHDError):
            s.set_boundary(8)
        M.lib().mhd_clear_error(s.h)
        s.set_state(st.U, st.B)
        s.set_boundary(3)
        with pytest.raises(M.MHDError):
            s.helicity()
        M.lib().mhd_clear_error(s.h)
        s.set_boundary(0)
        assert s.boundary() == 0
        s.helicity()
    finally:
        s.free()
