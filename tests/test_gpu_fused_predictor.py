"""The fused VL predictor (pencil-mask bit 3, k_vl_predictor): the
first-order fluxes of the three axes, the corner edge fields and the dt/2
update of Sec. 3.2's VL steps 1-3 in one kernel over 32 x 8-cell tiles
marched along z in chunks of 32 planes.

FP64 parity with the oracle at the 1e-12 bar, per field and step, on boxes
that fill whole tiles, on boxes whose x, y and z extents leave ragged tiles
and chunks, on boxes thinner than a tile's halo ring along every axis, and
on an uneven batch; FP32 and mixed agreement with the unfused predictor
(mask 7) after three steps at the bar of the other sweep-form comparisons;
launch counts and the cases where the bit is ignored (CTU, outflow)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1804_03479_b300 import inputs as I

pytestmark = pytest.mark.gpu

VL = [("vl", r, s) for r in ("plm", "ppm", "plm_prim") for s in ("roe", "hlld", "hlle")]


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


def parity(M, st, scheme, nsteps, mask=15, tol=1e-12):
    U, B = st.U.copy(), st.B.copy()
    s = M.Solver(U.shape[1:], st.dx, st.gamma, *scheme, "fp64", 0.3)
    try:
        s.set_sweep_pencils(mask, 32)
        assert s.launches_per_step() == 8
        for it in range(nsteps):
            s.set_state(U, B)
            dt = orc.cfl_dt(U, B, st.dx, st.gamma, 0.3)
            s.step(dt)
            orc.step(U, B, st.dx, st.gamma, dt, *scheme)
            Ug, Bg = s.get_state()
            for f in range(5):
                assert rel_l1(Ug[f], U[f]) <= tol, (scheme, it, f)
            for d in range(3):
                assert rel_l1(Bg[d], B[d]) <= tol, (scheme, it, d)
    finally:
        s.free()


@pytest.mark.parametrize("scheme", VL)
def test_fused_fp64_parity_whole_tiles(M, scheme):
    """64 x 32 x 64: two x tiles, four y tiles, two z chunks"""
    st = I.abc(None, kmult=1, beta=0.5, seed=11, noise=2e-2, shape=(64, 32, 64))
    parity(M, st, scheme, 2)


@pytest.mark.parametrize("shape", [(40, 20, 36), (33, 9, 65), (70, 17, 5)])
def test_fused_fp64_parity_ragged(M, shape):
    """tiles cut by the box along x and y, z chunks of 32 with a ragged last one"""
    st = I.abc(None, kmult=1, beta=0.5, seed=12, noise=3e-2, shape=shape)
    parity(M, st, ("vl", "plm", "roe"), 2)
    parity(M, st, ("vl", "ppm", "hlld"), 2)


@pytest.mark.parametrize("shape", [(1, 16, 16), (16, 1, 8), (9, 7, 1), (2, 3, 5)])
def test_fused_fp64_parity_thin_boxes(M, shape):
    """boxes thinner than the halo ring: the staged cells wrap several times"""
    L = shape[1] / 16.0
    st = I.abc(None, kmult=L, beta=0.5, seed=6, noise=5e-2, shape=shape, L=L)
    parity(M, st, ("vl", "ppm", "roe"), 2)
    parity(M, st, ("vl", "plm", "hlle"), 2)


def test_fused_fp64_parity_degenerate_states(M):
    """a field-aligned triple-point state and a B = 0 tube along each axis,
    each field's error over its natural scale (the transverse field starts
    at zero and the step creates it at second order)"""
    from test_gpu_degenerate import degenerate_state, scaled_errors
    from test_gpu_parity import TOL64
    for kind in ("field_aligned", "hydro"):
        for axis in range(3):
            st = degenerate_state(kind, axis, n=16)
            for solver in ("roe", "hlld", "hlle"):
                U, B = st.U.copy(), st.B.copy()
                s = M.Solver(U.shape[1:], st.dx, st.gamma, "vl", "plm", solver, "fp64", 0.3)
                try:
                    s.set_sweep_pencils(15, 32)
                    assert s.launches_per_step() == 8
                    s.set_state(U, B)
                    dt = orc.cfl_dt(U, B, st.dx, st.gamma, 0.3)
                    s.step(dt)
                    orc.step(U, B, st.dx, st.gamma, dt, "vl", "plm", solver)
                    Ug, Bg = s.get_state()
                    e = scaled_errors(Ug, Bg, U, B, st.gamma)
                    assert np.all(e <= TOL64), (kind, axis, solver, e)
                finally:
                    s.free()


def test_fused_fp64_batch_parity(M):
    """an uneven batch: every box's tiles in one launch, per-box dt"""
    boxes = [I.abc(16, kmult=1, beta=1.0, seed=21, noise=1e-2),
             I.abc(None, kmult=1, beta=0.5, seed=22, noise=3e-2, shape=(40, 12, 33)),
             I.orszag_tang(20, nz=6), I.linear_wave(12, "fast")]
    s = M.Solver(None, None, 5 / 3, "vl", "ppm", "roe", "fp64", 0.3,
                 shapes=[b.U.shape[1:] for b in boxes], dxs=[b.dx for b in boxes])
    try:
        s.set_sweep_pencils(15, 32)
        for k, b in enumerate(boxes):
            s.set_state(b.U, b.B, box=k)
        dts = np.array([orc.cfl_dt(b.U, b.B, b.dx, b.gamma, 0.3) for b in boxes])
        s.step(dts)
        for k, b in enumerate(boxes):
            U, B = b.U.copy(), b.B.copy()
            orc.step(U, B, b.dx, b.gamma, float(dts[k]), "vl", "ppm", "roe")
            Ug, Bg = s.get_state(box=k)
            mfloor = 1e-2 * np.abs(U[0]).sum()
            for f in range(5):
                den = max(np.abs(U[f]).sum(), mfloor if f in (1, 2, 3) else 0.0)
                assert np.abs(Ug[f] - U[f]).sum() / den <= 1e-12, (k, f)
            bfloor = 1e-2 * np.abs(B).sum() / 3
            for d in range(3):
                assert np.abs(Bg[d] - B[d]).sum() / max(np.abs(B[d]).sum(), bfloor) <= 1e-12, (k, d)
    finally:
        s.free()


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
@pytest.mark.parametrize("scheme", [("vl", "plm", "roe"), ("vl", "ppm", "hlld"), ("vl", "plm_prim", "hlle")])
def test_fused_agrees_with_sweeps(M, prec, scheme):
    """the same FP32 arithmetic per face in another kernel: rounding-level
    differences, grown over three steps"""
    st = I.abc(None, kmult=1, beta=0.5, seed=13, noise=2e-2, shape=(48, 24, 40))
    out = []
    for mask in (15, 7):
        s = M.Solver(st.U.shape[1:], st.dx, st.gamma, *scheme, prec, 0.3)
        try:
            s.set_sweep_pencils(mask, 32)
            cast = np.float32 if prec == "fp32" else np.float64     # the state exchange type
            s.set_state(st.U.astype(cast), st.B.astype(cast))
            s.advance(3)
            out.append(s.get_state())
        finally:
            s.free()
    (Ua, Ba), (Ub, Bb) = out
    for f in range(5):
        assert rel_l1(Ua[f].astype(np.float64), Ub[f].astype(np.float64)) <= 1e-5, (prec, f)
    for d in range(3):
        assert rel_l1(Ba[d].astype(np.float64), Bb[d].astype(np.float64)) <= 1e-5, (prec, d)


def test_fused_fp32_divergence_free(M):
    """CT through the fused kernel keeps div B at round-off (FP32 faces)"""
    st = I.abc(None, kmult=1, beta=0.5, seed=14, noise=2e-2, shape=(40, 24, 36))
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "ppm", "roe", "fp32", 0.3)
    try:
        s.set_state(st.U.astype(np.float32), st.B.astype(np.float32))
        s.advance(5)
        m, brms = s.divB()                           # max |div B| dx
        assert m <= 1e-5 * brms, (m, brms)
    finally:
        s.free()


def test_fused_bit_is_ignored_where_it_does_not_apply(M):
    st = I.abc(16, kmult=1, beta=0.5, seed=15)
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", "fp64", 0.3)
    try:
        assert s.sweep_pencils() == (23, 32)        # the FP64 default: the sweeps, x by staged pencils
        assert s.launches_per_step() == 12
        s.free()
        s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", "fp32", 0.3)
        assert s.sweep_pencils() == (743, 32)       # the FP32 VL PLM default: x by aligned marching warps,
        assert s.launches_per_step() == 11           # the half update in the y corrector, the
                                                     # conservative update in the z corrector
        s.set_sweep_pencils(15, 32)
        assert s.launches_per_step() == 8
        s.set_sweep_pencils(7, 32)
        assert s.launches_per_step() == 12
        s.set_sweep_pencils(15, 32)
        s.set_boundary(1)                            # an outflow axis: the sweeps run the predictor
        assert s.launches_per_step() == 12 + 2
    finally:
        s.free()
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "ctu", "plm", "roe", "fp64", 0.3)
    try:
        s.set_sweep_pencils(15, 32)
        assert s.launches_per_step() == 12
    finally:
        s.free()
