"""x by staged pencils (pencil-mask bit 4 with bit 0, k_xpencil): the VL
predictor and corrector sweeps along x with the lanes of a warp on 32
consecutive grid rows, cells and fluxes through per-warp shared-memory
chunks of 4 cells x 32 rows.

FP64 parity with the oracle at the 1e-12 bar per field and step: every VL
scheme; segment lengths that do and do not divide the rows, shorter than a
chunk and longer than the row; rows not a multiple of the chunk; boxes
whose row count leaves idle lanes in the last warp; thin boxes; outflow x
(the clamped lead-in of the first segment) and every outflow mask; an
uneven batch; with the unfused and the fused predictor.  FP32 and mixed
agreement with the x-warp form after three steps."""
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


def parity(M, U, B, dx, gam, scheme, mask, plen, nsteps, bc=0, tol=1e-12):
    U, B = U.copy(), B.copy()
    s = M.Solver(U.shape[1:], dx, gam, *scheme, "fp64", 0.3)
    try:
        if bc:
            s.set_boundary(bc)
        s.set_sweep_pencils(mask, plen)
        for it in range(nsteps):
            s.set_state(U, B)
            dt = orc.cfl_dt(U, B, dx, gam, 0.3, bc=bc) if bc else orc.cfl_dt(U, B, dx, gam, 0.3)
            s.step(dt)
            if bc:
                orc.step_bc(U, B, dx, gam, dt, *scheme, bc=bc)
            else:
                orc.step(U, B, dx, gam, dt, *scheme)
            Ug, Bg = s.get_state()
            for f in range(5):
                assert rel_l1(Ug[f], U[f]) <= tol, (scheme, mask, plen, bc, it, f)
            for d in range(3):
                assert rel_l1(Bg[d], B[d]) <= tol, (scheme, mask, plen, bc, it, d)
    finally:
        s.free()


@pytest.mark.parametrize("scheme", VL)
def test_xpencil_fp64_parity(M, scheme):
    st = I.abc(None, kmult=1, beta=0.5, seed=41, noise=2e-2, shape=(40, 24, 20))
    parity(M, st.U, st.B, st.dx, st.gamma, scheme, 23, 16, 2)


@pytest.mark.parametrize("plen", [3, 5, 7, 16, 32, 64])
def test_xpencil_fp64_parity_segment_lengths(M, plen):
    """nx = 37: segments that do and do not divide the rows, a last chunk
    of one to three cells, a segment longer than the row"""
    st = I.abc(None, kmult=1, beta=0.5, seed=42, noise=3e-2, shape=(37, 12, 10))
    parity(M, st.U, st.B, st.dx, st.gamma, ("vl", "plm", "roe"), 23, plen, 2)
    parity(M, st.U, st.B, st.dx, st.gamma, ("vl", "ppm", "hlld"), 23, plen, 2)


@pytest.mark.parametrize("shape", [(1, 16, 16), (2, 3, 5), (3, 9, 7), (16, 1, 8), (9, 7, 1)])
def test_xpencil_fp64_parity_thin_boxes(M, shape):
    """rows shorter than the stencil (the staged cells wrap several times),
    row counts that leave most lanes of the last warp idle"""
    L = shape[1] / 16.0
    st = I.abc(None, kmult=L, beta=0.5, seed=6, noise=5e-2, shape=shape, L=L)
    parity(M, st.U, st.B, st.dx, st.gamma, ("vl", "ppm", "roe"), 23, 4, 2)
    parity(M, st.U, st.B, st.dx, st.gamma, ("vl", "plm", "hlle"), 23, 16, 2)


@pytest.mark.parametrize("bc", [1, 3, 7])
@pytest.mark.parametrize("scheme", [("vl", "plm", "roe"), ("vl", "ppm", "hlld"), ("vl", "plm_prim", "hlle")])
def test_xpencil_fp64_parity_outflow(M, bc, scheme):
    st = I.open_box((26, 20, 18), seed=11)
    parity(M, st.U, st.B, st.dx, st.gamma, scheme, 23, 8, 2, bc=bc)


@pytest.mark.parametrize("scheme", [("vl", "plm", "roe"), ("vl", "ppm", "hlld")])
def test_xpencil_with_fused_predictor_fp64_parity(M, scheme):
    st = I.abc(None, kmult=1, beta=0.5, seed=43, noise=2e-2, shape=(48, 17, 33))
    parity(M, st.U, st.B, st.dx, st.gamma, scheme, 31, 32, 2)


def test_xpencil_fp64_batch_parity(M):
    boxes = [I.abc(16, kmult=1, beta=1.0, seed=21, noise=1e-2),
             I.abc(None, kmult=1, beta=0.5, seed=22, noise=3e-2, shape=(40, 12, 33)),
             I.orszag_tang(20, nz=6), I.linear_wave(12, "fast")]
    s = M.Solver(None, None, 5 / 3, "vl", "ppm", "roe", "fp64", 0.3,
                 shapes=[b.U.shape[1:] for b in boxes], dxs=[b.dx for b in boxes])
    try:
        s.set_sweep_pencils(23, 16)
        for k, b in enumerate(boxes):
            s.set_state(b.U, b.B, box=k)
        dts = np.array([orc.cfl_dt(b.U, b.B, b.dx, b.gamma, 0.3) for b in boxes])
        s.step(dts)
        for k, b in enumerate(boxes):
            U, B = b.U.copy(), b.B.copy()
            orc.step(U, B, b.dx, b.gamma, float(dts[k]), "vl", "ppm", "roe")
            Ug, Bg = s.get_state(box=k)
            # perturbation-size fields (the linear wave's momentum, the extruded
            # Orszag-Tang B_z): floors as in the batch tests
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
def test_xpencil_agrees_with_xwarps(M, prec, scheme):
    st = I.abc(None, kmult=1, beta=0.5, seed=44, noise=2e-2, shape=(48, 24, 40))
    cast = np.float32 if prec == "fp32" else np.float64
    out = []
    for mask in (23, 7):
        s = M.Solver(st.U.shape[1:], st.dx, st.gamma, *scheme, prec, 0.3)
        try:
            s.set_sweep_pencils(mask, 32)
            s.set_state(st.U.astype(cast), st.B.astype(cast))
            s.advance(3)
            out.append(s.get_state())
        finally:
            s.free()
    (Ua, Ba), (Ub, Bb) = out
    for f in range(5):
        assert rel_l1(Ua[f].astype(np.float64), Ub[f].astype(np.float64)) <= 1e-5, (prec, scheme, f)
    for d in range(3):
        assert rel_l1(Ba[d].astype(np.float64), Bb[d].astype(np.float64)) <= 1e-5, (prec, scheme, d)
