"""Edge-field staging (mhd_set_emf_staging): the planes of the edge-field
kernel (Sec. 2, Eqs. 13-14) staged by bulk tensor copies into a ring of
shared-memory slots, against per-thread loads.  Both forms compute the
same edges with the same arithmetic, so whole multi-step runs agree bit for
bit; the copied form is also held to the FP32 error statement against the
FP64 oracle.  Which contexts use which form, and argument checks.  (The
edge fields fused with their update, mode 2, are covered by
test_gpu_emf_update.py.)"""
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


def run(M, st, scheme, prec, mode, nsteps, bc=0):
    cast = np.float32 if prec == "fp32" else np.float64
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, *scheme, prec, 0.3)
    try:
        # the same sweep forms in both runs: the half update inside the y
        # corrector (mask bit 7, the FP32 / mixed PLM default) needs the
        # edge fields as their own kernel, so the copied form runs without it
        m, plen = s.sweep_pencils()
        s.set_sweep_pencils(m & 127, plen)
        s.set_emf_staging(mode)
        if bc:
            s.set_boundary(bc)
        s.set_state(st.U.astype(cast), st.B.astype(cast))
        s.advance(nsteps)
        U, B = s.get_state()
        return U, B, s.emf_staging()
    finally:
        s.free()


@pytest.mark.parametrize("shape,prec,scheme,bc", [
    ((64, 48, 40), "fp32", ("vl", "plm", "roe"), 0),
    ((44, 36, 20), "fp32", ("vl", "plm", "roe"), 0),       # ragged tiles on every axis
    ((44, 36, 20), "fp32", ("vl", "ppm", "hlld"), 7),      # outflow sides: the clamp at the lower halos
    ((64, 48, 33), "mixed", ("vl", "plm", "roe"), 0),
    ((44, 36, 20), "fp32", ("ctu", "plm", "roe"), 0),      # both stages' fluxes (F1, then F2)
    ((64, 9, 24), "fp32", ("ctu", "ppm", "hlld"), 5),      # one tile row, outflow on x and z
])
def test_tensor_copies_match_per_thread_loads_bitwise(M, shape, prec, scheme, bc):
    st = I.open_box(shape, seed=3) if bc else I.abc(0, kmult=1, beta=1.0, seed=1, shape=shape)
    U1, B1, (m1, a1) = run(M, st, scheme, prec, 1, 4, bc)
    U0, B0, (m0, a0) = run(M, st, scheme, prec, 0, 4, bc)
    assert (m1, a1) == (1, 1) and (m0, a0) == (0, 0)
    assert np.array_equal(U1, U0) and np.array_equal(B1, B0)


def test_tensor_copies_fp32_error_statement(M):
    """The copied form under the FP32 statement of the reduced-precision
    test (10 steps, same dt as the FP64 oracle), on a box it serves:
    relative L1 per field <= 1e-6 (rho, e, face B), 3e-4 (momentum, the
    1e-3 c_s noise)."""
    tol = np.array([1e-6, 3e-4, 3e-4, 3e-4, 1e-6, 1e-6, 1e-6, 1e-6])
    st = I.abc(0, kmult=1, beta=1.0, seed=0, shape=(44, 36, 20))
    U, B = st.U.copy(), st.B.copy()
    s = M.Solver(U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", "fp32", 0.3)
    try:
        s.set_emf_staging(1)
        assert s.emf_staging() == (1, 1)
        s.set_state(U.astype(np.float32), B.astype(np.float32))
        for _ in range(10):
            dt = orc.cfl_dt(U, B, st.dx, st.gamma, 0.3)
            s.step(dt)
            orc.step(U, B, st.dx, st.gamma, dt, "vl", "plm", "roe")
        Ug, Bg = s.get_state()
        errs = [rel_l1(Ug[f].astype(np.float64), U[f]) for f in range(5)] + \
               [rel_l1(Bg[d].astype(np.float64), B[d]) for d in range(3)]
        assert np.all(np.array(errs) <= tol), errs
        m, brms = s.divB()
        assert m / brms <= 1e-5
    finally:
        s.free()


@pytest.mark.parametrize("shape,prec,active", [
    ((64, 48, 40), "fp32", 1),
    ((64, 48, 40), "mixed", 1),
    ((64, 48, 40), "fp64", 0),    # 8-byte values: per-thread loads
    ((42, 48, 40), "fp32", 0),    # rows not a multiple of 16 bytes
    ((36, 48, 40), "fp32", 0),    # narrower than a staged plane
    ((64, 8, 40), "fp32", 0),     # fewer rows than a staged plane
])
def test_which_contexts_use_tensor_copies(M, shape, prec, active):
    nx, ny, nz = shape
    s = M.Solver((nz, ny, nx), 1.0 / ny, 5.0 / 3.0, "vl", "plm", "roe", prec, 0.3)
    try:
        assert s.emf_staging() == (0, 0)      # per-thread loads by default
        s.set_emf_staging(1)
        assert s.emf_staging() == (1, active)
        s.set_emf_staging(0)
        assert s.emf_staging() == (0, 0)
    finally:
        s.free()


def test_batches_use_per_thread_loads(M):
    s = M.Solver(None, 1.0 / 48, 5.0 / 3.0, "vl", "plm", "roe", "fp32", 0.3,
                 shapes=[(40, 48, 64), (40, 48, 64)])
    try:
        s.set_emf_staging(1)
        assert s.emf_staging() == (1, 0)
    finally:
        s.free()


def test_staging_arguments(M):
    s = M.Solver((40, 48, 64), 1.0 / 48, 5.0 / 3.0, "vl", "plm", "roe", "fp32", 0.3)
    try:
        for bad in (-1, 3):
            with pytest.raises(M.MHDError):
                s.set_emf_staging(bad)
            M.lib().mhd_clear_error(s.h)
        assert s.emf_staging() == (0, 0)
    finally:
        s.free()
