"""x by aligned marching warps (k_xmarch; pencil-mask bit 5 for the
predictor, bit 6 for the corrector, each with bit 0): the VL predictor and
PLM corrector sweeps along x, each warp marching a few grid rows back to
back, lane l of segment s on cell 32 s + l, the neighbours across the
segment ends from the previous segment's registers and the next segment's
prefetch, and each row's lead-in segment -1 in the corrector.

FP64 parity with the oracle at the 1e-12 bar per field and step: every VL
scheme (PPM: the predictor marches, the corrector keeps its x-warp); rows of
whole segments, ragged last segments, rows shorter than a segment (nx = 1:
every neighbour is the cell itself); outflow x (the clamped lead-in) and
every outflow mask; uneven batches whose boxes do not start on a segment
boundary and whose warps run from one box into the next.  FP32 and mixed agreement with the x-warp form after three steps;
the mask's range and precedence."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1804_03479_b300 import inputs as I

pytestmark = pytest.mark.gpu

VL = [("vl", r, s) for r in ("plm", "ppm", "plm_prim") for s in ("roe", "hlld", "hlle")]
MARCH = 103         # y / z pencils, x predictor and corrector by aligned marching warps


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


def parity(M, U, B, dx, gam, scheme, nsteps, bc=0, mask=MARCH, tol=1e-12):
    U, B = U.copy(), B.copy()
    s = M.Solver(U.shape[1:], dx, gam, *scheme, "fp64", 0.3)
    try:
        if bc:
            s.set_boundary(bc)
        s.set_sweep_pencils(mask, 32)
        per_axis = 2 if scheme[0] == "vl" else 1          # outer-face passes per outflow axis
        assert s.launches_per_step() == 12 + per_axis * bin(bc).count("1")
        for it in range(nsteps):
            s.set_state(U, B)
            dt = orc.cfl_dt(U, B, dx, gam, 0.3, bc=bc) if bc else orc.cfl_dt(U, B, dx, gam, 0.3)
            s.step(dt)
            if bc:
                orc.step_bc(U, B, dx, gam, dt, *scheme, bc=bc)
            else:
                orc.step(U, B, dx, gam, dt, *scheme)
            Ug, Bg = s.get_state()
            # momentum over a floor of 1e-2 of the density's sum: in the thin
            # ABC boxes it is a perturbation field (the batch tests' floor)
            mfloor = 1e-2 * np.abs(U[0]).sum()
            for f in range(5):
                den = max(np.abs(U[f]).sum(), mfloor if f in (1, 2, 3) else 0.0)
                assert np.abs(Ug[f] - U[f]).sum() / den <= tol, (scheme, bc, it, f)
            for d in range(3):
                assert rel_l1(Bg[d], B[d]) <= tol, (scheme, bc, it, d)
    finally:
        s.free()


@pytest.mark.parametrize("scheme", VL)
def test_xmarch_fp64_parity_whole_segments(M, scheme):
    """nx = 64: two segments a row, both stencil ends across a segment boundary"""
    st = I.abc(None, kmult=1, beta=0.5, seed=51, noise=2e-2, shape=(64, 12, 10))
    parity(M, st.U, st.B, st.dx, st.gamma, scheme, 2)


@pytest.mark.parametrize("shape", [(40, 12, 8), (33, 9, 6), (31, 5, 7), (96, 8, 6)])
def test_xmarch_fp64_parity_ragged(M, shape):
    """a last segment of 8, 1 or 31 cells (its wrapped lanes feed the
    stencil), three whole segments"""
    st = I.abc(None, kmult=1, beta=0.5, seed=52, noise=3e-2, shape=shape)
    parity(M, st.U, st.B, st.dx, st.gamma, ("vl", "plm", "roe"), 2)
    parity(M, st.U, st.B, st.dx, st.gamma, ("vl", "plm_prim", "hlld"), 2)


@pytest.mark.parametrize("shape", [(1, 16, 16), (2, 3, 5), (5, 9, 7), (16, 1, 8), (9, 7, 1)])
def test_xmarch_fp64_parity_short_rows(M, shape):
    """rows shorter than a segment: the lanes' cells wrap several times"""
    L = shape[1] / 16.0
    st = I.abc(None, kmult=L, beta=0.5, seed=6, noise=5e-2, shape=shape, L=L)
    parity(M, st.U, st.B, st.dx, st.gamma, ("vl", "plm", "hlle"), 2)
    parity(M, st.U, st.B, st.dx, st.gamma, ("vl", "ppm", "roe"), 2)


@pytest.mark.parametrize("bc", [1, 3, 7])
@pytest.mark.parametrize("scheme", [("vl", "plm", "roe"), ("vl", "ppm", "hlld"), ("vl", "plm_prim", "hlle")])
def test_xmarch_fp64_parity_outflow(M, bc, scheme):
    """outflow x: the lead-in segment and the next-segment prefetch clamp"""
    st = I.open_box((26, 20, 18), seed=11)
    parity(M, st.U, st.B, st.dx, st.gamma, scheme, 2, bc=bc)


def test_xmarch_fp64_parity_outflow_whole_segments(M):
    """nx = 64 with outflow x: the last segment's lane 31 takes the clamped
    cell from the prefetch of segment 2"""
    st = I.open_box((64, 10, 8), seed=12)
    parity(M, st.U, st.B, st.dx, st.gamma, ("vl", "plm", "roe"), 2, bc=1)


def test_xmarch_fp64_batch_parity(M):
    """an uneven batch: box offsets that are not multiples of 32 cells"""
    boxes = [I.abc(16, kmult=1, beta=1.0, seed=21, noise=1e-2),
             I.abc(None, kmult=1, beta=0.5, seed=22, noise=3e-2, shape=(40, 12, 33)),
             I.orszag_tang(20, nz=6), I.linear_wave(12, "fast")]
    s = M.Solver(None, None, 5 / 3, "vl", "plm", "roe", "fp64", 0.3,
                 shapes=[b.U.shape[1:] for b in boxes], dxs=[b.dx for b in boxes])
    try:
        s.set_sweep_pencils(MARCH, 32)
        for k, b in enumerate(boxes):
            s.set_state(b.U, b.B, box=k)
        dts = np.array([orc.cfl_dt(b.U, b.B, b.dx, b.gamma, 0.3) for b in boxes])
        s.step(dts)
        for k, b in enumerate(boxes):
            U, B = b.U.copy(), b.B.copy()
            orc.step(U, B, b.dx, b.gamma, float(dts[k]), "vl", "plm", "roe")
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


@pytest.mark.parametrize("scheme", [("vl", "plm", "roe"), ("vl", "plm_prim", "hlld")])
def test_xmarch_fp64_batch_warps_cross_boxes(M, scheme):
    """row counts (15, 21, 25, 9) that are not multiples of a warp's rows:
    warps whose rows run from one box into the next, with another x length,
    offset and periodic wrap"""
    shapes = [(16, 3, 5), (33, 7, 3), (40, 5, 5), (70, 3, 3)]
    boxes = [I.abc(None, kmult=1, beta=0.5, seed=60 + k, noise=3e-2, shape=sh) for k, sh in enumerate(shapes)]
    s = M.Solver(None, None, 5 / 3, *scheme, "fp64", 0.3,
                 shapes=[b.U.shape[1:] for b in boxes], dxs=[b.dx for b in boxes])
    try:
        s.set_sweep_pencils(MARCH, 32)
        for k, b in enumerate(boxes):
            s.set_state(b.U, b.B, box=k)
        dts = np.array([orc.cfl_dt(b.U, b.B, b.dx, b.gamma, 0.3) for b in boxes])
        s.step(dts)
        for k, b in enumerate(boxes):
            U, B = b.U.copy(), b.B.copy()
            orc.step(U, B, b.dx, b.gamma, float(dts[k]), *scheme)
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
@pytest.mark.parametrize("scheme", [("vl", "plm", "roe"), ("vl", "plm", "hlld"), ("vl", "plm_prim", "hlle"),
                                    ("vl", "ppm", "roe")])
def test_xmarch_agrees_with_xwarps(M, prec, scheme):
    """the same per-face arithmetic in another kernel: rounding-level
    differences, grown over three steps"""
    st = I.abc(None, kmult=1, beta=0.5, seed=54, noise=2e-2, shape=(64, 24, 40))
    cast = np.float32 if prec == "fp32" else np.float64
    out = []
    for mask in (MARCH, 7):                          # the marching warps against the overlapping ones
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


CTU = [("ctu", r, s) for r in ("plm", "ppm") for s in ("roe", "hlld", "hlle")]   # (PLM_PRIM: VL only)


@pytest.mark.parametrize("scheme", CTU)
def test_xmarch_ctu_tracing_fp64_parity(M, scheme):
    """CTU steps 1-2 along x by the march (mask bit 5): traced states with
    the dB_n/dn source from the shifted face field, written per cell, and
    their fluxes (PPM: the x-warps)"""
    st = I.abc(None, kmult=1, beta=0.5, seed=57, noise=2e-2, shape=(64, 12, 10))
    parity(M, st.U, st.B, st.dx, st.gamma, scheme, 2, mask=39)


@pytest.mark.parametrize("shape", [(40, 12, 8), (33, 9, 6), (5, 9, 7), (1, 16, 16)])
def test_xmarch_ctu_tracing_fp64_parity_ragged_and_short(M, shape):
    L = shape[1] / 16.0
    st = I.abc(None, kmult=L, beta=0.5, seed=58, noise=3e-2, shape=shape, L=L)
    parity(M, st.U, st.B, st.dx, st.gamma, ("ctu", "plm", "roe"), 2, mask=39)
    parity(M, st.U, st.B, st.dx, st.gamma, ("ctu", "plm", "hlld"), 2, mask=39)


@pytest.mark.parametrize("bc", [1, 6])
def test_xmarch_ctu_fp64_parity_outflow(M, bc):
    """an outflow x keeps the tile sweep along x (its lead-in is cell 0 with
    its own stencil); outflow y / z with x periodic marches"""
    st = I.open_box((26, 20, 18), seed=13)
    parity(M, st.U, st.B, st.dx, st.gamma, ("ctu", "plm", "roe"), 2, bc=bc, mask=39)


def test_xmarch_ctu_fp64_batch_parity(M):
    """uneven boxes, per-box dt and dx in the traced states"""
    shapes = [(16, 3, 5), (33, 7, 3), (40, 5, 5), (70, 3, 3)]
    boxes = [I.abc(None, kmult=1, beta=0.5, seed=70 + k, noise=3e-2, shape=sh) for k, sh in enumerate(shapes)]
    scheme = ("ctu", "plm", "hlle")
    s = M.Solver(None, None, 5 / 3, *scheme, "fp64", 0.3,
                 shapes=[b.U.shape[1:] for b in boxes], dxs=[b.dx for b in boxes])
    try:
        s.set_sweep_pencils(39, 32)
        for k, b in enumerate(boxes):
            s.set_state(b.U, b.B, box=k)
        dts = np.array([orc.cfl_dt(b.U, b.B, b.dx, b.gamma, 0.3) for b in boxes])
        s.step(dts)
        for k, b in enumerate(boxes):
            U, B = b.U.copy(), b.B.copy()
            orc.step(U, B, b.dx, b.gamma, float(dts[k]), *scheme)
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
@pytest.mark.parametrize("scheme", [("ctu", "plm", "roe"), ("ctu", "plm", "hlld"), ("ctu", "plm", "hlle")])
def test_xmarch_ctu_agrees_with_xwarps(M, prec, scheme):
    st = I.abc(None, kmult=1, beta=0.5, seed=59, noise=2e-2, shape=(64, 24, 40))
    cast = np.float32 if prec == "fp32" else np.float64
    out = []
    for mask in (39, 7):
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


def test_xmarch_fp32_divergence_free(M):
    st = I.abc(None, kmult=1, beta=0.5, seed=55, noise=2e-2, shape=(64, 24, 36))
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", "fp32", 0.3)
    try:
        s.set_sweep_pencils(MARCH, 32)
        s.set_state(st.U.astype(np.float32), st.B.astype(np.float32))
        s.advance(5)
        m, brms = s.divB()
        assert m <= 1e-5 * brms, (m, brms)
    finally:
        s.free()


def test_xmarch_mask_range_and_precedence(M):
    st = I.abc(16, kmult=1, beta=0.5, seed=15)
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", "fp64", 0.3)
    try:
        assert s.sweep_pencils() == (23, 32)        # FP64 VL: x by staged pencils
        s.set_sweep_pencils(127, 32)
        assert s.sweep_pencils() == (127, 32)
        with pytest.raises(M.MHDError):
            s.set_sweep_pencils(1024, 32)
        M.lib().mhd_clear_error(s.h)
        assert s.sweep_pencils() == (127, 32)
    finally:
        s.free()
    for prec, scheme, mask in [("fp32", ("vl", "plm", "roe"), 743), ("fp32", ("vl", "plm_prim", "hlle"), 743),
                               ("fp32", ("vl", "ppm", "hlld"), 743), ("mixed", ("vl", "plm", "roe"), 487),
                               ("fp32", ("ctu", "plm", "roe"), 679), ("fp64", ("ctu", "plm", "roe"), 39)]:
        s = M.Solver(st.U.shape[1:], st.dx, st.gamma, *scheme, prec, 0.3)
        try:
            assert s.sweep_pencils() == (mask, 32), (prec, scheme)
        finally:
            s.free()
    # bits 5 and 6 without bit 0: x stays on tiles; with bit 4: x by staged
    # pencils; bit 6 alone: the corrector marches, the predictor keeps its warps
    for mask in (102, 55, 119, 71):
        parity(M, st.U, st.B, st.dx, st.gamma, ("vl", "plm", "roe"), 1, mask=mask)
