"""mhd_step_noalloc, the step for callers that may not allocate device memory
(a plug-in whose host application owns all device memory, or a loop that
cannot afford cudaMalloc's device-wide synchronisation).  It must give the
same state as the ordinary context-based step, call after call, although
its scratch is one fixed array shared by every call.

Named to be collected last, so that a run stopping at the first failure has
run every other test before this one."""
import ctypes

import numpy as np
import pytest

from paper_1804_03479_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_03479_b300 import mhd
    mhd.lib()
    return torch, mhd


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


@pytest.mark.parametrize("recon,riemann,n", [("ppm", "hlld", 24), ("plm", "roe", 32)])
def test_noalloc_matches_context_step_twice(env, recon, riemann, n):
    torch, mhd = env
    st = I.abc(n, kmult=1, beta=1.0, seed=3, noise=1e-2)
    # the ordinary entry points: a context that owns its scratch
    s = mhd.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", recon, riemann, "fp64", 0.3)
    s.set_state(st.U, st.B)
    dts, ref = [], []
    for _ in range(2):
        dt = s.cfl_dt()
        s.step(dt)
        dts.append(dt)
        ref.append(s.get_state())
    s.free()
    # the allocation-free step on a caller-owned device state, two calls in a row
    U = torch.from_numpy(st.U).cuda()
    B = torch.from_numpy(st.B).cuda()
    torch.cuda.synchronize()
    for k in range(2):
        mhd.step_noalloc(U, B, st.dx, dts[k], st.gamma, recon, riemann)
        torch.cuda.synchronize()
        Ug, Bg = U.cpu().numpy(), B.cpu().numpy()
        Ur, Br = ref[k]
        for f in range(5):
            assert rel_l1(Ug[f], Ur[f]) <= 1e-12, (k, f)
        for d in range(3):
            assert rel_l1(Bg[d], Br[d]) <= 1e-12, (k, d)


def test_noalloc_rejects_what_it_cannot_hold(env):
    torch, mhd = env
    st = I.abc(40, kmult=1)          # 64000 cells > the 32768-cell scratch
    U = torch.from_numpy(st.U).cuda()
    B = torch.from_numpy(st.B).cuda()
    with pytest.raises(mhd.MHDError) as ei:
        mhd.step_noalloc(U, B, st.dx, 1e-3, st.gamma)
    assert ei.value.status == mhd.MHD_EINVAL
    assert "exceed" in str(ei.value)
    small = I.abc(8, kmult=1)
    U = torch.from_numpy(small.U).cuda()
    B = torch.from_numpy(small.B).cuda()
    g = mhd.Grid(8, 8, 8, small.dx)
    s = mhd.Scheme(1, 0, 0, 0, 0.3)   # CTU is not built for this entry point
    st_ = mhd.lib().mhd_step_noalloc(ctypes.byref(g), small.gamma, ctypes.byref(s), 1e-3,
                                     ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(B.data_ptr()), None)
    assert st_ == mhd.MHD_EUNSUPPORTED
