"""Each precision's step as the first thing a process runs.

The FP32, mixed and learned steps are compiled in separate units that each
hold their own instance of the edge-field kernel, whose shared memory exceeds
the default 48 KB limit.  A limit raised on one unit's instance does not
cover another's, so a process whose first context is mixed must step as well
as one that created an FP32 context before.  The child process runs two
steps of one scheme in a fresh interpreter; the parent runs the same steps
after every other test of this module has created its contexts, and the two
results must agree bit for bit (the kernels are deterministic).
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from paper_1804_03479_b300 import inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys
    import numpy as np
    sys.path.insert(0, {root!r})
    from paper_1804_03479_b300 import inputs as I
    from paper_1804_03479_b300 import mhd
    st = I.abc(32, kmult=1, beta=1.0, seed=0)
    cast = np.float32 if {prec!r} == "fp32" else np.float64
    s = mhd.Solver(st.U.shape[1:], st.dx, st.gamma, {integ!r}, "plm", "roe", {prec!r}, 0.3)
    s.set_state(st.U.astype(cast), st.B.astype(cast))
    s.advance(2)
    s.sync()
    U, B = s.get_state()
    s.free()
    np.savez({out!r}, U=U, B=B)
""")


def run_in_parent(prec, integ):
    from paper_1804_03479_b300 import mhd
    st = I.abc(32, kmult=1, beta=1.0, seed=0)
    cast = np.float32 if prec == "fp32" else np.float64
    s = mhd.Solver(st.U.shape[1:], st.dx, st.gamma, integ, "plm", "roe", prec, 0.3)
    try:
        s.set_state(st.U.astype(cast), st.B.astype(cast))
        s.advance(2)
        s.sync()
        return s.get_state()
    finally:
        s.free()


@pytest.fixture(scope="module")
def warm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    # contexts of every precision in this process first
    for p in ("fp32", "fp64", "mixed"):
        run_in_parent(p, "vl")


@pytest.mark.parametrize("prec,integ", [("mixed", "vl"), ("mixed", "ctu"), ("fp32", "vl"), ("fp64", "vl")])
def test_first_context_of_a_process_steps(warm, tmp_path, prec, integ):
    out = str(tmp_path / "state.npz")
    code = CHILD.format(root=ROOT, prec=prec, integ=integ, out=out)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    child = np.load(out)
    U, B = run_in_parent(prec, integ)
    assert np.array_equal(child["U"], U) and np.array_equal(child["B"], B)
