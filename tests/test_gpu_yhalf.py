"""Per-cell passes inside the VL step's y pencils.

The primitives at t^n and the CFL signal speeds inside the first-order y
predictor pencils (k_yprim; pencil-mask bit 8 with bit 1): each pencil
thread forms the primitives of its segment's cells and one lead-in cell,
stores its own cells', folds their signal speeds into the box maximum
(device dt) and solves its y faces.

The conservative part of the full update inside the corrector's z pencils
(k_zfull; pencil-mask bit 9 with bit 2), the face field by CT alone after
the edge fields (k_ct, k_ct4).

The VL half update fused into the corrector's y pencils (k_yhalf;
pencil-mask bit 7 with bit 1): each pencil thread forms the half-step state
(Sec. 3.2 VL step 3: Eq. 13 for the faces, Eq. 10 with dt/2 for the cells,
Eq. 5 for the primitives) of every cell its PLM walk reconstructs, stores
the half-step primitives and faces of the cells it owns and the y fluxes;
the x and z corrector sweeps, the corrector's edge fields and the full
update then read the corrector fluxes from the second flux array.

The per-cell arithmetic is the half-update kernel's and the per-face
arithmetic the PLM pencil's; the compiler may form fused multiply-adds
differently in the two kernels, so the fused step agrees with the separate
kernels' to rounding (FP64 at the 1e-12 parity bar, FP32 and mixed within
1e-5 after three steps, as other kernel forms of the same arithmetic).
FP64 parity with the oracle at the 1e-12 bar covers the whole step on
whole, ragged and short lines, segment lengths down to one face (every
lead-in cell owned by another segment) and uneven batches; the pressure
floor is checked against the separate kernels.  FP32 and mixed PLM
contexts take bit 7 by default."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1804_03479_b300 import inputs as I

pytestmark = pytest.mark.gpu

PLM = [("vl", r, s) for r in ("plm", "plm_prim") for s in ("roe", "hlld", "hlle")]
FUSED64, FUSED32 = 23 | 128, 103 | 128     # the precision defaults with bit 7
PRIM = 256                                   # bit 8
ZFULL = 512                                  # bit 9


@pytest.fixture(scope="module")
def M():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_03479_b300 import mhd
    mhd.lib()
    return mhd


def parity(M, st, scheme, nsteps, mask=FUSED64, plen=32, pfloor=0.0, tol=1e-12, device_dt=False):
    """FP64 steps against the oracle from the same state; with device_dt
    the library's own CFL dt (the signal speeds of the primitive pass), held
    to 1e-14 of the oracle's"""
    U, B = st.U.copy(), st.B.copy()
    s = M.Solver(U.shape[1:], st.dx, st.gamma, *scheme, "fp64", 0.3, pfloor=pfloor)
    try:
        s.set_sweep_pencils(mask, plen)
        fused = bool(mask & 128) + bool(mask & PRIM and not pfloor)
        assert s.launches_per_step() == 12 - fused
        for it in range(nsteps):
            s.set_state(U, B)
            dt = orc.cfl_dt(U, B, st.dx, st.gamma, 0.3, pfloor=pfloor) if pfloor else \
                orc.cfl_dt(U, B, st.dx, st.gamma, 0.3)
            if device_dt:
                s.advance(1)
                dtg = s.last_dt()
                assert abs(dtg - dt) <= 1e-14 * dt, (dtg, dt)
                dt = dtg
            else:
                s.step(dt)
            if pfloor:
                orc.step_floor(U, B, st.dx, st.gamma, dt, *scheme, pfloor=pfloor)
            else:
                orc.step(U, B, st.dx, st.gamma, dt, *scheme)
            Ug, Bg = s.get_state()
            # momentum over a floor of 1e-2 of the density's sum (perturbation
            # fields in the thin boxes), as the other parity tests
            mfloor = 1e-2 * np.abs(U[0]).sum()
            for f in range(5):
                den = max(np.abs(U[f]).sum(), mfloor if f in (1, 2, 3) else 0.0)
                assert np.abs(Ug[f] - U[f]).sum() / den <= tol, (scheme, it, f)
            for d in range(3):
                den = np.abs(B[d]).sum()
                assert np.abs(Bg[d] - B[d]).sum() / (den if den > 0 else 1.0) <= tol, (scheme, it, d)
    finally:
        s.free()


VL = [("vl", r, s) for r in ("plm", "ppm", "plm_prim") for s in ("roe", "hlld", "hlle")]


@pytest.mark.parametrize("scheme", PLM + [("vl", "ppm", s) for s in ("roe", "hlld", "hlle")])
def test_zfull_fp64_parity(M, scheme):
    """bit 9 alone, and with bits 7 and 8 (the corrector fluxes in the second
    array), against the oracle"""
    st = I.abc(None, kmult=1, beta=0.5, seed=89, noise=2e-2, shape=(64, 10, 12))
    parity(M, st, scheme, 2, mask=23 | ZFULL)
    parity(M, st, scheme, 2, mask=23 | ZFULL | 128 | PRIM, device_dt=True)


@pytest.mark.parametrize("shape", [(40, 8, 12), (33, 6, 9), (2, 5, 9), (1, 9, 7), (3, 3, 1), (36, 6, 20)])
@pytest.mark.parametrize("plen", [1, 3, 32])
def test_zfull_fp64_parity_ragged_short(M, shape, plen):
    """last segments of 8 and 1 faces, lines of 1-3 cells, 16-byte aligned
    and unaligned rows (the CT kernel's quads and single cells); the box
    length from ny, as the other ragged cases"""
    L = max(shape[1], 1) / 16.0
    st = I.abc(None, kmult=L, beta=0.5, seed=90, noise=3e-2, shape=shape, L=L)
    parity(M, st, ("vl", "plm", "roe"), 2, mask=23 | ZFULL | 128, plen=plen)
    parity(M, st, ("vl", "ppm", "hlld"), 2, mask=23 | ZFULL, plen=plen)


def test_zfull_fp64_batch(M):
    shapes = [(16, 5, 3), (33, 3, 7), (40, 5, 5), (70, 3, 3), (5, 2, 1)]
    boxes = [I.abc(None, kmult=1, beta=0.5, seed=100 + k, noise=3e-2, shape=sh) for k, sh in enumerate(shapes)]
    scheme = ("vl", "plm_prim", "hlle")
    s = M.Solver(None, None, 5 / 3, *scheme, "fp64", 0.3,
                 shapes=[b.U.shape[1:] for b in boxes], dxs=[b.dx for b in boxes])
    try:
        s.set_sweep_pencils(23 | ZFULL | 128 | PRIM, 8)
        for k, b in enumerate(boxes):
            s.set_state(b.U, b.B, box=k)
        s.advance(1)
        dts = s.last_dts()
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
@pytest.mark.parametrize("scheme", [("vl", "plm", "roe"), ("vl", "plm_prim", "hlld"), ("vl", "ppm", "hlld")])
def test_zfull_agrees_with_the_full_update(M, prec, scheme):
    """three graph-replayed steps with bits 7, 8 and 9 against the separate
    kernels (quad-aligned box and a 33-wide one)"""
    for shape in [(40, 48, 64), (20, 12, 33)]:
        st = I.abc(None, kmult=1, beta=0.5, seed=91, noise=2e-2, shape=shape)
        agree(M, st, prec, scheme, 3, extra=ZFULL)


@pytest.mark.parametrize("scheme", VL)
def test_yprim_fp64_parity_device_dt(M, scheme):
    """bit 8 alone and with bit 7: the device dt from the pencils' signal
    speeds and the whole step against the oracle"""
    st = I.abc(None, kmult=1, beta=0.5, seed=86, noise=2e-2, shape=(10, 64, 12))
    parity(M, st, scheme, 2, mask=23 | PRIM, device_dt=True)
    parity(M, st, scheme, 2, mask=23 | PRIM | 128, device_dt=True)


@pytest.mark.parametrize("shape", [(8, 40, 12), (6, 33, 9), (5, 2, 9), (9, 1, 7), (3, 3, 1)])
@pytest.mark.parametrize("plen", [1, 3, 32])
def test_yprim_fp64_parity_ragged_short(M, shape, plen):
    L = max(shape[1], 1) / 16.0
    st = I.abc(None, kmult=L, beta=0.5, seed=87, noise=3e-2, shape=shape, L=L)
    parity(M, st, ("vl", "plm", "roe"), 2, mask=23 | PRIM | 128, plen=plen, device_dt=True)


def test_yprim_fp64_batch_device_dt(M):
    """uneven boxes: each box's dt from its own signal-speed maximum, warps
    whose lanes run from one box into the next"""
    shapes = [(5, 16, 3), (3, 33, 7), (5, 40, 5), (3, 70, 3), (2, 5, 1)]
    boxes = [I.abc(None, kmult=1, beta=0.5, seed=95 + k, noise=3e-2, shape=sh) for k, sh in enumerate(shapes)]
    scheme = ("vl", "plm", "hlld")
    s = M.Solver(None, None, 5 / 3, *scheme, "fp64", 0.3,
                 shapes=[b.U.shape[1:] for b in boxes], dxs=[b.dx for b in boxes])
    try:
        s.set_sweep_pencils(23 | PRIM | 128, 8)
        for k, b in enumerate(boxes):
            s.set_state(b.U, b.B, box=k)
        s.advance(1)
        dts = s.last_dts()
        for k, b in enumerate(boxes):
            dto = orc.cfl_dt(b.U, b.B, b.dx, b.gamma, 0.3)
            assert abs(dts[k] - dto) <= 1e-14 * dto, (k, dts[k], dto)
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


def test_yprim_reports_a_negative_pressure(M):
    """the anomaly record (MHD_ENEGATIVE with the first bad cell) from the
    fused primitive pass"""
    st = I.abc(16, kmult=1, beta=0.5, seed=88)
    U, B = st.U.copy(), st.B.copy()
    U[4, 3, 5, 7] = -1.0                               # energy below the magnetic and kinetic parts
    s = M.Solver(U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", "fp64", 0.3)
    try:
        s.set_sweep_pencils(23 | PRIM, 32)
        s.set_state(U, B)
        s.advance(1)
        with pytest.raises(M.MHDError) as ei:
            s.sync()
        assert ei.value.status == M.MHD_ENEGATIVE
        assert s.bad_cell() == (3 * 16 + 5) * 16 + 7
    finally:
        s.free()


@pytest.mark.parametrize("scheme", VL)
def test_yhalf_fp64_parity(M, scheme):
    """ny = 64: two segments a line, lead-ins and look-ahead across them"""
    st = I.abc(None, kmult=1, beta=0.5, seed=81, noise=2e-2, shape=(10, 64, 12))
    parity(M, st, scheme, 2)


@pytest.mark.parametrize("shape", [(8, 40, 12), (6, 33, 9), (7, 31, 5), (5, 2, 9), (9, 1, 7), (3, 3, 1)])
def test_yhalf_fp64_parity_ragged_and_short(M, shape):
    """a last segment of 8, 1 or 31 faces; lines shorter than the stencil
    (ny = 1, 2, 3: every lead-in and look-ahead cell wraps onto the line)"""
    L = max(shape[1], 1) / 16.0
    st = I.abc(None, kmult=L, beta=0.5, seed=82, noise=3e-2, shape=shape, L=L)
    parity(M, st, ("vl", "plm", "roe"), 2)
    parity(M, st, ("vl", "plm_prim", "hlld"), 2, mask=FUSED32)
    parity(M, st, ("vl", "ppm", "hlle"), 2)


@pytest.mark.parametrize("plen", [1, 2, 3, 5])
def test_yhalf_fp64_parity_short_segments(M, plen):
    """segments of 1-5 faces: every cell is also formed, unstored, by the
    lead-ins of one or two other segments"""
    st = I.abc(None, kmult=1, beta=0.5, seed=83, noise=2e-2, shape=(6, 23, 10))
    parity(M, st, ("vl", "plm", "hlle"), 2, plen=plen)
    parity(M, st, ("vl", "ppm", "roe"), 2, plen=plen)


def agree(M, st, prec, scheme, nsteps, pfloor=0.0, extra=0):
    """the same steps with and without bit 7 (graph-replayed), per-field
    relative L1 of the difference; returns the two floor counts"""
    cast = np.float32 if prec == "fp32" else np.float64
    base = 23 if prec == "fp64" else 103
    out, floors, dts = [], [], []
    for mask in (base, base | 128 | (0 if pfloor else PRIM) | extra):
        s = M.Solver(st.U.shape[1:], st.dx, st.gamma, *scheme, prec, 0.3, pfloor=pfloor)
        try:
            s.set_sweep_pencils(mask, 32)
            s.set_state(st.U.astype(cast), st.B.astype(cast))
            s.advance(nsteps, use_graph=True)
            out.append(s.get_state())
            floors.append(s.floor_count())
            dts.append(s.last_dt())
        finally:
            s.free()
    (Ua, Ba), (Ub, Bb) = out
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert abs(dts[0] - dts[1]) <= (1e-14 if prec == "fp64" else 1e-6) * dts[0], dts
    for f in range(5):
        a, b = Ua[f].astype(np.float64), Ub[f].astype(np.float64)
        den = max(np.abs(b).sum(), 1e-2 * np.abs(Ub[0]).sum() if f in (1, 2, 3) else 0.0)
        assert np.abs(a - b).sum() / den <= tol, (prec, scheme, f)
    for d in range(3):
        a, b = Ba[d].astype(np.float64), Bb[d].astype(np.float64)
        assert np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300) <= tol, (prec, scheme, d)
    return floors


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
def test_yhalf_pressure_floor(M, prec):
    """a floor above the blast's ambient pressure binds at the start of the
    step and in the half-step primitives: the fused walk applies it as the
    separate half update does.  (Against the oracle the static ambient
    medium's mass fluxes are zero up to rounding, and the edge fields'
    upwinding by their sign is then a rounding-level decision: after one
    fused step the hydrodynamic fields agreed at 1e-12, B_x to 4.4e-7.)"""
    fa, fb = agree(M, I.mhd_blast(24), prec, ("vl", "plm", "hlld"), 2, pfloor=2e-2)
    assert fa == fb and fa > 0


def test_yhalf_fp64_batch_parity(M):
    """uneven boxes, per-box dt: lines of several lengths and offsets"""
    shapes = [(5, 16, 3), (3, 33, 7), (5, 40, 5), (3, 70, 3)]
    boxes = [I.abc(None, kmult=1, beta=0.5, seed=90 + k, noise=3e-2, shape=sh) for k, sh in enumerate(shapes)]
    scheme = ("vl", "plm", "roe")
    s = M.Solver(None, None, 5 / 3, *scheme, "fp64", 0.3,
                 shapes=[b.U.shape[1:] for b in boxes], dxs=[b.dx for b in boxes])
    try:
        s.set_sweep_pencils(FUSED64, 32)
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


@pytest.mark.parametrize("prec", ["fp32", "mixed", "fp64"])
@pytest.mark.parametrize("scheme", VL)
def test_yhalf_agrees_with_separate_kernels(M, prec, scheme):
    """three graph-replayed steps with and without bit 7"""
    st = I.abc(None, kmult=1, beta=0.5, seed=84, noise=2e-2, shape=(40, 48, 64))
    agree(M, st, prec, scheme, 3)


def test_mask_range_defaults_and_fallbacks(M):
    """bits 7 to 9 are accepted up to 1023; bits 7 and 9 are the FP32 PLM
    default, bit 7 the FP32 PPM default, bits 7 and 8 the mixed PLM default,
    bit 8 the mixed PPM default; with
    PPM (bit 9), a pressure floor (bit 8), outflow boundaries or without
    bit 1 the separate kernels run"""
    st = I.abc(16, kmult=1, beta=0.5, seed=85)
    for prec, recon, mask, nl in [("fp32", "plm", FUSED32 | ZFULL, 11), ("fp32", "ppm", FUSED32 | ZFULL, 11),
                                  ("mixed", "plm_prim", FUSED32 | PRIM, 10), ("mixed", "ppm", 103 | PRIM, 11),
                                  ("fp64", "plm", 23, 12)]:
        s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", recon, "roe", prec, 0.3)
        try:
            assert s.sweep_pencils() == (mask, 32), (prec, recon)
            assert s.launches_per_step() == nl, (prec, recon)
        finally:
            s.free()
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", "fp32", 0.3)
    try:
        s.set_sweep_pencils(511, 32)
        assert s.sweep_pencils() == (511, 32)
        assert s.launches_per_step() == 8          # bit 3, the fused predictor, takes precedence
        s.set_sweep_pencils(FUSED32 | PRIM, 32)
        assert s.launches_per_step() == 10
        s.set_sweep_pencils((FUSED32 | PRIM) & ~2, 32)   # y by tiles: neither y pencil takes a pass
        assert s.launches_per_step() == 12
        with pytest.raises(M.MHDError):
            s.set_sweep_pencils(1024, 32)
        M.lib().mhd_clear_error(s.h)
        s.set_sweep_pencils(FUSED32 | PRIM, 32)
        s.set_boundary(2)                          # outflow y
        assert s.launches_per_step() == 12 + 2
    finally:
        s.free()
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "ppm", "roe", "fp32", 0.3)
    try:
        s.set_sweep_pencils(FUSED32 | PRIM | ZFULL, 32)
        assert s.launches_per_step() == 10         # (bit 9: the same count)
    finally:
        s.free()
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", "mixed", 0.3, pfloor=1e-6)
    try:
        assert s.sweep_pencils() == (FUSED32 | PRIM, 32)
        assert s.launches_per_step() == 11         # a pressure floor: the primitive pass of its own
    finally:
        s.free()


CTU = [("ctu", r, s) for r in ("plm", "ppm") for s in ("roe", "hlld", "hlle")]


@pytest.mark.parametrize("scheme", CTU)
def test_ctu_yhalf_fp64_parity(M, scheme):
    """CTU with bit 7 (k_ctu_yhalf): the dt/2 update inside the y pencils of
    the transverse correction, against the oracle"""
    st = I.abc(None, kmult=1, beta=0.5, seed=110, noise=2e-2, shape=(12, 64, 10))
    parity(M, st, scheme, 2, mask=39 | 128)
    parity(M, st, scheme, 2, mask=39 | 128, device_dt=True)


@pytest.mark.parametrize("scheme", CTU)
def test_ctu_zfull_fp64_parity(M, scheme):
    """CTU with bit 9 (k_ctu_zfull): the conservative update inside the z
    pencils of the transverse correction, alone and with bit 7"""
    st = I.abc(None, kmult=1, beta=0.5, seed=113, noise=2e-2, shape=(12, 10, 64))
    parity(M, st, scheme, 2, mask=39 | ZFULL)
    parity(M, st, scheme, 2, mask=39 | 128 | ZFULL, device_dt=True)


@pytest.mark.parametrize("shape", [(8, 40, 12), (6, 33, 9), (5, 2, 9), (9, 1, 7), (3, 3, 1)])
@pytest.mark.parametrize("plen", [1, 32])
def test_ctu_yhalf_fp64_parity_ragged_short(M, shape, plen):
    L = max(shape[1], 1) / 16.0
    st = I.abc(None, kmult=L, beta=0.5, seed=111, noise=3e-2, shape=shape, L=L)
    parity(M, st, ("ctu", "plm", "roe"), 2, mask=39 | 128, plen=plen)
    st = I.abc(None, kmult=L, beta=0.5, seed=114, noise=3e-2, shape=(shape[0], shape[2], shape[1]), L=L)
    parity(M, st, ("ctu", "ppm", "hlle"), 2, mask=39 | 128 | ZFULL, plen=plen)


def test_ctu_yhalf_fp64_batch(M):
    shapes = [(5, 16, 3), (3, 33, 7), (5, 40, 5), (3, 70, 3)]
    boxes = [I.abc(None, kmult=1, beta=0.5, seed=120 + k, noise=3e-2, shape=sh) for k, sh in enumerate(shapes)]
    scheme = ("ctu", "ppm", "hlld")
    s = M.Solver(None, None, 5 / 3, *scheme, "fp64", 0.3,
                 shapes=[b.U.shape[1:] for b in boxes], dxs=[b.dx for b in boxes])
    try:
        s.set_sweep_pencils(39 | 128 | ZFULL, 16)
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
@pytest.mark.parametrize("scheme", [("ctu", "plm", "roe"), ("ctu", "ppm", "hlld")])
def test_ctu_yhalf_agrees_with_separate_kernels(M, prec, scheme):
    st = I.abc(None, kmult=1, beta=0.5, seed=112, noise=2e-2, shape=(40, 48, 64))
    cast = np.float32 if prec == "fp32" else np.float64
    out = []
    for mask in (39, 39 | 128 | ZFULL):
        s = M.Solver(st.U.shape[1:], st.dx, st.gamma, *scheme, prec, 0.3)
        try:
            s.set_sweep_pencils(mask, 32)
            assert s.launches_per_step() == (11 if mask & 128 else 12)
            s.set_state(st.U.astype(cast), st.B.astype(cast))
            s.advance(3, use_graph=True)
            out.append(s.get_state())
        finally:
            s.free()
    (Ua, Ba), (Ub, Bb) = out
    for f in range(5):
        a, b = Ua[f].astype(np.float64), Ub[f].astype(np.float64)
        den = max(np.abs(a).sum(), 1e-2 * np.abs(Ua[0]).sum() if f in (1, 2, 3) else 0.0)
        assert np.abs(a - b).sum() / den <= 1e-5, (prec, scheme, f)
    for d in range(3):
        a, b = Ba[d].astype(np.float64), Bb[d].astype(np.float64)
        assert np.abs(a - b).sum() / np.abs(a).sum() <= 1e-5, (prec, scheme, d)
