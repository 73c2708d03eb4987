"""Pencil sweeps (mhd_set_sweep_pencils): one thread per segment of
consecutive faces along the sweep axis (VL: x by warps), for the VL
predictor and corrector and the CTU tracing sweeps.  FP64 parity with the
oracle at the 1e-12 bar on cubic, ragged and thin boxes, segment lengths
that do and do not divide the lines, and the tile sweeps everywhere
(mask 0); agreement with the tile sweeps; argument checks."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1804_03479_b300 import inputs as I

pytestmark = pytest.mark.gpu

VL = [("vl", r, s) for r in ("plm", "ppm", "plm_prim") for s in ("roe", "hlld", "hlle")]
CTU = [("ctu", r, s) for r in ("plm", "ppm") for s in ("roe", "hlld", "hlle")]


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


def parity(M, st, scheme, mask, plen, nsteps, tol=1e-12):
    U, B = st.U.copy(), st.B.copy()
    s = M.Solver(U.shape[1:], st.dx, st.gamma, *scheme, "fp64", 0.3)
    try:
        s.set_sweep_pencils(mask, plen)
        assert s.sweep_pencils() == (mask, plen)
        for it in range(nsteps):
            s.set_state(U, B)
            dt = orc.cfl_dt(U, B, st.dx, st.gamma, 0.3)
            s.step(dt)
            orc.step(U, B, st.dx, st.gamma, dt, *scheme)
            Ug, Bg = s.get_state()
            for f in range(5):
                assert rel_l1(Ug[f], U[f]) <= tol, (scheme, mask, plen, it, f)
            for d in range(3):
                assert rel_l1(Bg[d], B[d]) <= tol, (scheme, mask, plen, it, d)
    finally:
        s.free()


@pytest.mark.parametrize("scheme", VL)
def test_pencil_fp64_parity_abc32(M, scheme):
    st = I.abc(32, kmult=1, beta=1.0, seed=0)
    parity(M, st, scheme, 7, 16, 4)


@pytest.mark.parametrize("scheme", CTU)
@pytest.mark.parametrize("mask,plen", [(7, 16), (6, 5), (1, 7)])
def test_ctu_tracing_pencils_fp64_parity(M, scheme, mask, plen):
    st = I.abc(None, kmult=1, beta=0.5, seed=6, noise=3e-2, shape=(24, 20, 18))
    parity(M, st, scheme, mask, plen, 3)


@pytest.mark.parametrize("scheme", [("ctu", "plm", "roe"), ("ctu", "ppm", "hlld"), ("ctu", "plm", "hlle")])
def test_ctu_xwarp_tracing_fp64_parity_long_rows(M, scheme):
    """CTU tracing by warps along x over several warp segments per row
    (nx = 70: 29 + 29 + 12 faces for PLM, 27 + 27 + 16 for PPM)"""
    st = I.abc(None, kmult=1, beta=0.5, seed=7, noise=3e-2, shape=(70, 12, 10))
    parity(M, st, scheme, 7, 16, 3)


@pytest.mark.parametrize("mask,plen", [(0, 16), (7, 5), (6, 32), (1, 7), (7, 64)])
def test_pencil_fp64_parity_ragged(M, mask, plen):
    st = I.abc(None, kmult=1, beta=0.5, seed=5, noise=3e-2, shape=(40, 24, 20))
    parity(M, st, ("vl", "plm", "roe"), mask, plen, 2)
    parity(M, st, ("vl", "ppm", "hlld"), mask, plen, 2)


@pytest.mark.parametrize("shape", [(1, 16, 16), (16, 1, 8), (9, 7, 1), (2, 3, 5)])
def test_pencil_fp64_parity_thin_boxes(M, shape):
    L = shape[1] / 16.0
    st = I.abc(None, kmult=L, beta=0.5, seed=6, noise=5e-2, shape=shape, L=L)
    parity(M, st, ("vl", "ppm", "roe"), 7, 3, 2)
    parity(M, st, ("vl", "plm", "hlld"), 7, 16, 2)


@pytest.mark.parametrize("prec", ["fp32", "fp64", "mixed"])
def test_pencils_agree_with_tiles_on_a_batch(M, prec):
    boxes = [I.abc(16, kmult=1, beta=1.0, seed=21, noise=1e-2), I.linear_wave(12, "fast"),
             I.abc(None, kmult=1, beta=0.5, seed=22, noise=3e-2, shape=(24, 16, 8)),
             I.orszag_tang(20, nz=6)]
    cast = np.float32 if prec == "fp32" else np.float64
    out = []
    for mask in (0, 7, 6, 15, 23):
        s = M.Solver(None, None, 5 / 3, "vl", "ppm", "hlld", prec, 0.3,
                     shapes=[b.U.shape[1:] for b in boxes], dxs=[b.dx for b in boxes])
        try:
            if mask:
                s.set_sweep_pencils(mask, 8)
            for k, b in enumerate(boxes):
                s.set_state(b.U.astype(cast), b.B.astype(cast), box=k)
            s.advance(3)
            out.append([s.get_state(box=k) for k in range(len(boxes))])
        finally:
            s.free()
    # FP64: the same arithmetic; FP32 sweeps (FP32 and mixed forms): rounding-level
    # differences of the two kernels' code, grown over three PPM/HLLD steps
    tol = {"fp64": 1e-13, "mixed": 1e-5, "fp32": 1e-5}[prec]
    for other in out[1:]:
        for k, ((Ua, Ba), (Ub, Bb)) in enumerate(zip(out[0], other)):
            # the momentum of the 1e-6 linear wave is itself a perturbation:
            # its denominator is floored at 1e-2 sum|rho|
            mfloor = 1e-2 * np.abs(Ua[0].astype(np.float64)).sum()
            for f in range(5):
                a, b = Ub[f].astype(np.float64), Ua[f].astype(np.float64)
                den = max(np.abs(b).sum(), mfloor if f in (1, 2, 3) else 0.0)
                assert np.abs(a - b).sum() / den <= tol, (prec, k, f)
            # likewise a B component that vanishes in exact arithmetic (B_z of the
            # extruded Orszag-Tang box): floor at 1e-2 of the mean component
            bfloor = 1e-2 * np.abs(Ba.astype(np.float64)).sum() / 3
            for d in range(3):
                a, b = Bb[d].astype(np.float64), Ba[d].astype(np.float64)
                assert np.abs(a - b).sum() / max(np.abs(b).sum(), bfloor) <= tol, (prec, k, d)


def test_pencil_arguments(M):
    st = I.abc(8, kmult=1, beta=1.0)
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", "fp64", 0.3)
    try:
        for mask, plen in [(1024, 16), (-1, 16), (7, 0), (7, 2000)]:
            with pytest.raises(M.MHDError):
                s.set_sweep_pencils(mask, plen)
            lib = M.lib()
            lib.mhd_clear_error(s.h)
    finally:
        s.free()
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "ctu", "plm", "roe", "fp64", 0.3)
    try:
        assert s.sweep_pencils() == (39, 32)      # the CTU default: x tracing by aligned marching warps, pencils on y and z
        s.set_sweep_pencils(6, 16)
        assert s.sweep_pencils() == (6, 16)
    finally:
        s.free()


def test_autotune_considers_pencils_and_keeps_results(M):
    st = I.abc(48, kmult=2, beta=0.5, seed=3)
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", "fp64", 0.3)
    try:
        s.set_state(st.U, st.B)
        tl, bps, ms = s.autotune(reps=1)
        mask, plen = s.sweep_pencils()
        assert mask in (0, 6, 7, 23, 103, 15, 31, 111, 151, 231, 359, 487, 743, 999) and plen in (8, 16, 32) and ms > 0
        U, B = st.U.copy(), st.B.copy()
        Ug, Bg = s.get_state()
        assert np.array_equal(Ug, U) and np.array_equal(Bg, B)   # state restored
        dt = orc.cfl_dt(U, B, st.dx, st.gamma, 0.3)
        s.step(dt)
        orc.step(U, B, st.dx, st.gamma, dt, "vl", "plm", "roe")
        Ug, Bg = s.get_state()
        for f in range(5):
            assert rel_l1(Ug[f], U[f]) <= 1e-12
    finally:
        s.free()
