"""The 1-D Riemann problems of Table 1 (Sec. 5.1 (ii)) through the whole
scheme of the oracle, on periodic lines holding the problem and its mirror
image.  The exact (Torrilhon) solutions are not available, so the pins are
what holds without them: positive density and pressure, exact conservation
on the periodic line, the normal field left constant, and self-convergence of
the profiles under refinement (first order or better across
discontinuities)."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1804_03479_b300 import inputs as I

GOLDEN = __file__.replace("test_oracle_shocktubes.py", "golden/table1_riemann_states.txt")
T_END = {"torrilhon": 0.1, "rj2a": 0.12}


def table1():
    rows = {}
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            vals = [float(eval(t, {"math": math})) for t in tok[1:]]
            rows[tok[0]] = (np.array(vals[0:7]), np.array(vals[7:14]), vals[14])
    return rows


def run(name, n, scheme, axis=0):
    wl, wr, bn = table1()[name]
    st = I.shock_tube(wl, wr, bn, n, axis=axis, m=1)
    U, B = st.U.copy(), st.B.copy()
    t, T = 0.0, T_END[name]
    s0 = orc.sums(U, B)
    while t < T:
        dt = min(orc.cfl_dt(U, B, st.dx, st.gamma, 0.3), T - t)
        orc.step(U, B, st.dx, st.gamma, dt, *scheme)
        t += dt
    return st, U, B, s0


@pytest.mark.parametrize("name", ["torrilhon", "rj2a"])
@pytest.mark.parametrize("scheme", [("vl", "plm", "roe"), ("vl", "ppm", "hlld"), ("ctu", "plm", "hlld"),
                                    ("ctu", "ppm", "roe"), ("vl", "plm", "hlle")])
def test_table1_tubes_positive_and_conservative(name, scheme):
    st, U, B, s0 = run(name, 256, scheme)
    W = orc.prim(U, B, st.gamma)
    assert np.all(np.isfinite(U)) and np.all(np.isfinite(B))
    assert W[0].min() > 0 and W[4].min() > 0
    s1 = orc.sums(U, B)
    scale = np.array([np.abs(st.U[f]).sum() for f in range(5)] + [np.abs(st.B[d]).sum() for d in range(3)])
    assert np.all(np.abs(s1 - s0) <= 1e-13 * scale + 1e-13)
    # the normal field of a 1-D problem stays at its value
    assert np.abs(B[0] - st.B[0]).max() <= 1e-13


@pytest.mark.parametrize("name", ["torrilhon", "rj2a"])
def test_table1_tubes_self_convergence(name):
    scheme = ("vl", "plm", "roe")
    prof = {}
    for n in (128, 256, 512, 1024):
        st, U, B, _ = run(name, n, scheme)
        prof[n] = orc.prim(U, B, st.gamma)[:, 0, 0, :]
    def diff(n):
        # the n profile against the 2n profile averaged to n cells, in the window
        # around the problem at 3L/4
        fine = 0.5 * (prof[2 * n][:, 0::2] + prof[2 * n][:, 1::2])
        x = (np.arange(n) + 0.5) / n * 2.0
        sel = (x > 1.0) & (x < 2.0)
        return np.abs(prof[n][:, sel] - fine[:, sel]).mean(axis=1)
    d128, d256, d512 = diff(128), diff(256), diff(512)
    for f in (0, 4, 6, 7):   # rho, P, B_y, B_z (the transverse field of a tube along x)
        assert d256[f] < d128[f] and d512[f] < d256[f], (name, f, d128[f], d256[f], d512[f])
        # two refinements: 4x at first order; the rotating transverse field of
        # the Torrilhon problem (the test's point: a rotation resolved only at
        # high resolution) converges slowest, so the bound is loose
        assert d128[f] / d512[f] > 1.5, (name, f, d128[f] / d512[f])


def test_tube_axes_agree():
    """the same problem along x, y and z gives the same profile (relabelled), to
    rounding: the three axes' operations are the same up to their order"""
    scheme = ("vl", "ppm", "hlld")
    out = []
    for axis in range(3):
        st, U, B, _ = run("rj2a", 128, scheme, axis=axis)
        W = orc.prim(U, B, st.gamma)
        t1, t2 = (axis + 1) % 3, (axis + 2) % 3
        line = [W[0], W[1 + axis], W[1 + t1], W[1 + t2], W[4], W[5 + t1], W[5 + t2]]
        out.append(np.stack([a.reshape(-1) for a in line]))
    for k in (1, 2):
        assert np.abs(out[k] - out[0]).max() <= 1e-10 * (1 + np.abs(out[0]).max())
