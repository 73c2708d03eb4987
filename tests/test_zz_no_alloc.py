"""mhd_step_noalloc, the step for callers that may not allocate device memory
(a plug-in whose host application owns all device memory, or a loop that
cannot afford cudaMalloc's device-wide synchronisation).  It must give the
same state as the ordinary context-based step, call after call, although
its scratch is one fixed array shared by every call, and it must not take
any device memory after its first call.

Named to be collected last, so that a run stopping at the first failure has
run every other test before this one."""
import ctypes

import numpy as np
import pytest

from paper_1804_03479_b300 import inputs as I

TOL = 1e-12   # relative L1 per field, the FP64 parity bar of the other tests


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_03479_b300 import mhd
    mhd.lib()
    return torch, mhd


def _context_steps(mhd, st, recon, riemann, pfloor, nsteps=2):
    """The ordinary entry points: a context that owns its scratch."""
    s = mhd.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", recon, riemann, "fp64", 0.3, pfloor=pfloor)
    s.set_state(st.U, st.B)
    dts, ref = [], []
    for _ in range(nsteps):
        dt = s.cfl_dt()
        s.step(dt)
        dts.append(dt)
        ref.append(s.get_state())
    if pfloor > 0.0:
        assert s.floor_count() > 0     # the floor binds: the case tests something
    s.free()
    return dts, ref


def _noalloc_matches(torch, mhd, st, recon, riemann, pfloor=0.0):
    dts, ref = _context_steps(mhd, st, recon, riemann, pfloor)
    U = torch.from_numpy(st.U).cuda()
    B = torch.from_numpy(st.B).cuda()
    torch.cuda.synchronize()
    free_after_first = None
    for k in range(2):
        mhd.step_noalloc(U, B, st.dx, dts[k], st.gamma, recon, riemann, pfloor=pfloor)
        torch.cuda.synchronize()
        if k == 0:
            free_after_first = torch.cuda.mem_get_info()[0]
        else:
            # the second call takes no device memory (the first may load the
            # library's device code and reserve its array)
            assert torch.cuda.mem_get_info()[0] == free_after_first
        Ug, Bg = U.cpu().numpy(), B.cpu().numpy()
        Ur, Br = ref[k]
        for f in range(5):
            assert rel_l1(Ug[f], Ur[f]) <= TOL, (k, f)
        for d in range(3):
            assert rel_l1(Bg[d], Br[d]) <= TOL, (k, d)


@pytest.mark.gpu
@pytest.mark.parametrize("riemann", ["roe", "hlld", "hlle"])
@pytest.mark.parametrize("recon", ["plm", "ppm", "plm_prim"])
def test_noalloc_matches_context_step_twice(env, recon, riemann):
    torch, mhd = env
    st = I.abc(24, kmult=1, beta=1.0, seed=3, noise=1e-2)
    _noalloc_matches(torch, mhd, st, recon, riemann)


@pytest.mark.gpu
def test_noalloc_non_cubic_box_below_one_tile(env):
    """6 x 12 x 20 cells: a side below the sweep tile's 8 cells."""
    torch, mhd = env
    st = I.open_box((6, 12, 20), seed=4)
    _noalloc_matches(torch, mhd, st, "ppm", "hlld")
    _noalloc_matches(torch, mhd, st, "plm", "roe")


@pytest.mark.gpu
def test_noalloc_pressure_floor_as_context_step(env):
    """With pfloor > 0 the energy raise at the step start and the floored
    half-step pressure are those of mhd_step.  The floor sits 0.1 % below the
    uniform initial pressure; the 1e-2 c_s velocity noise moves P by about
    1.6 %, so the half step of the first call and the start of the second
    fall below it."""
    torch, mhd = env
    st = I.abc(16, kmult=1, beta=1.0, seed=5, noise=1e-2)
    P0 = st.meta["P0"]
    _noalloc_matches(torch, mhd, st, "plm", "roe", pfloor=P0 * 0.999)


@pytest.mark.gpu
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


@pytest.mark.parametrize("sides", [(1 << 21, 1 << 21, 1 << 22), (1 << 30, 1 << 30, 1 << 30),
                                   (32769, 1, 1), (1, 1, 32769), (182, 181, 1)])
def test_noalloc_rejects_wrapping_cell_counts_on_the_host(sides):
    """Grids whose cell count would wrap a 64-bit product (2^21 x 2^21 x 2^22
    wraps to 0) or just exceeds the scratch are refused before any launch:
    no device is needed."""
    from paper_1804_03479_b300 import mhd
    g = mhd.Grid(*sides, 1.0)
    s = mhd.Scheme(0, 0, 0, 0, 0.3)
    dummy = ctypes.c_void_p(16)     # never dereferenced: the call returns first
    st = mhd.lib().mhd_step_noalloc(ctypes.byref(g), 5.0 / 3.0, ctypes.byref(s), 1e-3, dummy, dummy, None)
    assert st == mhd.MHD_EINVAL
    assert b"exceed" in mhd.lib().mhd_last_error(None)


def test_init_rejects_wrapping_cell_counts_on_the_host():
    """mhd_init bounds the cell count (< 2^31 per box) without a wrapping
    product, before touching the device."""
    from paper_1804_03479_b300 import mhd
    L = mhd.lib()
    s = mhd.Scheme(0, 0, 0, 0, 0.3)
    for sides in [(1 << 21, 1 << 21, 1 << 22), (1 << 30, 1 << 30, 4), (1 << 16, 1 << 15, 1)]:
        g = mhd.Grid(*sides, 1.0)
        out = ctypes.c_void_p()
        st = L.mhd_init(ctypes.byref(g), 5.0 / 3.0, ctypes.byref(s), None, ctypes.byref(out))
        assert st == mhd.MHD_EINVAL, sides
        assert not out.value
