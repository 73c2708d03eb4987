"""Error plumbing and checkpoint/resume through the C ABI.

- A bounded device wait that gives up sets the context's wait flag; the next
  call that reads the device flags must return MHD_ETIMEOUT (not a generic
  CUDA error), the error stays until mhd_clear_error, and the context stays
  usable.  The flag is written from the host (mhd_inject_wait_flag): no wait
  on the GPU is made to fail.
- Resume: N steps straight must equal, bit for bit, N/2 steps, a copy of the
  state out (mhd_get_state), a new context seeded with it (mhd_set_state) and
  N/2 more steps.  The step has no hidden state beyond U and the face B (dt
  is recomputed from the state each step).
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("bits", [1, 2, 3])
def test_wait_flag_reports_timeout(M, bits):
    st = I.abc(16, kmult=1, beta=1.0, seed=1)
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", "fp32", 0.3)
    try:
        s.set_state(st.U.astype(np.float32), st.B.astype(np.float32))
        s.advance(1)
        s.sync()
        s.inject_wait_flag(bits)
        for call in (s.sync, s.cfl_dt, s.sums):
            with pytest.raises(M.MHDError) as ei:
                call()
            assert ei.value.status == M.MHD_ETIMEOUT, call
            assert "gave up" in str(ei.value)
        s.clear_error()
        s.sync()
        s.advance(2)
        s.sync()
        U, _ = s.get_state()
        assert np.isfinite(U).all()
    finally:
        s.free()


def test_wait_flag_injection_rejects_bad_bits(M):
    st = I.abc(8, kmult=1)
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma)
    try:
        for bad in (0, 4, 255):
            with pytest.raises(M.MHDError) as ei:
                s.inject_wait_flag(bad)
            assert ei.value.status == M.MHD_EINVAL
    finally:
        s.free()


CASES = [("vl", "plm", "roe", "fp64"), ("ctu", "ppm", "hlld", "fp64"), ("vl", "plm", "roe", "fp32"),
         ("ctu", "plm", "hlle", "fp32"), ("vl", "ppm", "hlld", "mixed"), ("ctu", "plm", "roe", "mixed")]


@pytest.mark.parametrize("integ,recon,solver,prec", CASES)
@pytest.mark.parametrize("graph", [False, True])
def test_resume_is_bitwise(M, integ, recon, solver, prec, graph):
    N = 8
    st = I.abc(40, kmult=2, beta=0.5, seed=11, noise=1e-2)
    dtype = np.float32 if prec == "fp32" else np.float64   # MIXED state is passed as double
    U0, B0 = st.U.astype(dtype), st.B.astype(dtype)

    def ctx():
        return M.Solver(st.U.shape[1:], st.dx, st.gamma, integ, recon, solver, prec, 0.3)

    a = ctx()
    try:
        a.set_state(U0, B0)
        a.advance(N, use_graph=graph)
        Ua, Ba = a.get_state()
    finally:
        a.free()
    b = ctx()
    try:
        b.set_state(U0, B0)
        b.advance(N // 2, use_graph=graph)
        Uh, Bh = b.get_state()       # the checkpoint
    finally:
        b.free()
    c = ctx()
    try:
        c.set_state(Uh, Bh)          # resumed in a fresh context
        c.advance(N - N // 2, use_graph=graph)
        Uc, Bc = c.get_state()
    finally:
        c.free()
    assert np.array_equal(Ua, Uc) and np.array_equal(Ba, Bc)
    assert not np.array_equal(Ua, U0.astype(Ua.dtype))   # the steps did something

