"""The edge fields fused with the update that uses them (mhd_set_emf_staging
mode 2, opt-in; k_emf_update): per 32 x 8-cell tile marched along z, the corner
edge fields of Eqs. 13-14 in shared memory, then the dt/2 update to
B^{n+1/2} and the half-step primitives (VL steps 2-3, CTU steps 3-4) or the
full update (VL steps 6-7, CTU steps 7-8).

FP64 parity with the oracle at the 1e-12 bar per field and step (mode 2 on
request; VL and CTU, every solver, with and without the fused predictor),
on boxes that leave ragged tiles and z chunks, on thin boxes and on an
uneven batch; FP32 and mixed agreement with the separate kernels (mode 0)
after three steps; div B at round-off; launch counts; outflow contexts fall
back to the separate kernels."""
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


def parity(M, st, scheme, nsteps, mask=7, tol=1e-12):
    U, B = st.U.copy(), st.B.copy()
    s = M.Solver(U.shape[1:], st.dx, st.gamma, *scheme, "fp64", 0.3)
    try:
        s.set_emf_staging(2)
        s.set_sweep_pencils(mask, 32)
        assert s.emf_staging() == (2, 2)
        for it in range(nsteps):
            s.set_state(U, B)
            dt = orc.cfl_dt(U, B, st.dx, st.gamma, 0.3)
            s.step(dt)
            orc.step(U, B, st.dx, st.gamma, dt, *scheme)
            Ug, Bg = s.get_state()
            for f in range(5):
                assert rel_l1(Ug[f], U[f]) <= tol, (scheme, mask, it, f)
            for d in range(3):
                assert rel_l1(Bg[d], B[d]) <= tol, (scheme, mask, it, d)
    finally:
        s.free()


SCHEMES = [(i, r, s) for i in ("vl", "ctu") for r in ("plm", "ppm") for s in ("roe", "hlld", "hlle")]


@pytest.mark.parametrize("scheme", SCHEMES)
def test_emf_update_fp64_parity(M, scheme):
    st = I.abc(None, kmult=1, beta=0.5, seed=31, noise=2e-2, shape=(40, 20, 36))
    parity(M, st, scheme, 2)


@pytest.mark.parametrize("scheme", [("vl", "plm", "roe"), ("vl", "ppm", "hlld"), ("vl", "plm_prim", "hlle")])
def test_emf_update_with_fused_predictor_fp64_parity(M, scheme):
    """every edge field of the step in shared memory: the predictor's (fused
    predictor) and the corrector's (fused with the full update)"""
    st = I.abc(None, kmult=1, beta=0.5, seed=32, noise=2e-2, shape=(33, 17, 40))
    parity(M, st, scheme, 2, mask=15)


@pytest.mark.parametrize("shape", [(1, 16, 16), (16, 1, 8), (9, 7, 1), (2, 3, 5)])
def test_emf_update_fp64_parity_thin_boxes(M, shape):
    L = shape[1] / 16.0
    st = I.abc(None, kmult=L, beta=0.5, seed=6, noise=5e-2, shape=shape, L=L)
    parity(M, st, ("vl", "ppm", "roe"), 2)
    parity(M, st, ("ctu", "plm", "hlld"), 2)


def test_emf_update_fp64_batch_parity(M):
    boxes = [I.abc(16, kmult=1, beta=1.0, seed=21, noise=1e-2),
             I.abc(None, kmult=1, beta=0.5, seed=22, noise=3e-2, shape=(40, 12, 33)),
             I.orszag_tang(20, nz=6), I.linear_wave(12, "fast")]
    for integ in ("vl", "ctu"):
        s = M.Solver(None, None, 5 / 3, integ, "plm", "hlld", "fp64", 0.3,
                     shapes=[b.U.shape[1:] for b in boxes], dxs=[b.dx for b in boxes])
        try:
            s.set_emf_staging(2)
            for k, b in enumerate(boxes):
                s.set_state(b.U, b.B, box=k)
            dts = np.array([orc.cfl_dt(b.U, b.B, b.dx, b.gamma, 0.3) for b in boxes])
            s.step(dts)
            for k, b in enumerate(boxes):
                U, B = b.U.copy(), b.B.copy()
                orc.step(U, B, b.dx, b.gamma, float(dts[k]), integ, "plm", "hlld")
                Ug, Bg = s.get_state(box=k)
                # the 1e-6 linear wave's momentum and the extruded Orszag-Tang
                # B_z are perturbation-size fields: floors as in the batch tests
                mfloor = 1e-2 * np.abs(U[0]).sum()
                for f in range(5):
                    den = max(np.abs(U[f]).sum(), mfloor if f in (1, 2, 3) else 0.0)
                    assert np.abs(Ug[f] - U[f]).sum() / den <= 1e-12, (integ, k, f)
                bfloor = 1e-2 * np.abs(B).sum() / 3
                for d in range(3):
                    assert np.abs(Bg[d] - B[d]).sum() / max(np.abs(B[d]).sum(), bfloor) <= 1e-12, (integ, k, d)
        finally:
            s.free()


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
@pytest.mark.parametrize("scheme", [("vl", "plm", "roe"), ("vl", "ppm", "hlld"), ("ctu", "plm", "roe"),
                                    ("ctu", "ppm", "hlle")])
def test_emf_update_agrees_with_separate_kernels(M, prec, scheme):
    st = I.abc(None, kmult=1, beta=0.5, seed=33, noise=2e-2, shape=(48, 24, 40))
    cast = np.float32 if prec == "fp32" else np.float64
    out = []
    for mode in (2, 0):
        s = M.Solver(st.U.shape[1:], st.dx, st.gamma, *scheme, prec, 0.3)
        try:
            s.set_emf_staging(mode)
            assert s.emf_staging() == (mode, mode)
            s.set_state(st.U.astype(cast), st.B.astype(cast))
            s.advance(3)
            out.append(s.get_state())
            if mode == 2:
                m, brms = s.divB()
                assert m <= 1e-5 * brms, (m, brms)
        finally:
            s.free()
    (Ua, Ba), (Ub, Bb) = out
    for f in range(5):
        assert rel_l1(Ua[f].astype(np.float64), Ub[f].astype(np.float64)) <= 1e-5, (prec, scheme, f)
    for d in range(3):
        assert rel_l1(Ba[d].astype(np.float64), Bb[d].astype(np.float64)) <= 1e-5, (prec, scheme, d)


def test_emf_update_launch_counts_and_fallbacks(M):
    st = I.abc(16, kmult=1, beta=0.5, seed=15)
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", "fp32", 0.3)
    try:
        assert s.emf_staging() == (0, 0) and s.sweep_pencils()[0] == 743
        s.set_sweep_pencils(15, 32)
        assert s.launches_per_step() == 8
        s.set_emf_staging(2)
        assert s.emf_staging() == (2, 2)
        assert s.launches_per_step() == 7            # prim, dt, predictor, 3 sweeps, edge fields + full update
        s.set_sweep_pencils(7, 32)
        assert s.launches_per_step() == 10
        s.set_emf_staging(0)
        assert s.launches_per_step() == 12
        s.set_emf_staging(2)
        s.set_boundary(2)                            # an outflow axis: the separate kernels
        assert s.emf_staging() == (2, 0) and s.launches_per_step() == 12 + 2
    finally:
        s.free()
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "ctu", "plm", "roe", "mixed", 0.3)
    try:
        s.set_emf_staging(2)
        assert s.emf_staging() == (2, 2) and s.launches_per_step() == 10
    finally:
        s.free()
