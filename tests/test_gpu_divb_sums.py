"""mhd_divB (Eq. 16) and mhd_sums (Sec. 5.1 (v)) against the oracle's
orc_divB / orc_sums, value by value, on the same state.

The oracle's two functions are pinned to closed forms in
tests/test_oracle_divb_sums.py; here the GPU reductions (per-virtual-block
partials folded in a fixed order per box) must give the same numbers:

- the per-cell divergence is the same three FP64 differences added in the
  same order on both sides, so max|div B| dx must agree bit for bit;
- the sums and B_rms are FP64 sums in a different order: both lie within
  (n-1) u sum|x| of the exact sum (u = 2^-53), so they may differ by at most
  twice that (the rigorous bound for any two summation orders);
- integer-valued fields sum exactly in any order: equality.
The boxes have ragged cell counts (not multiples of the 256-cell virtual
block), and a batch checks each box separately, so a reduction that dropped
the last partial block, or mixed boxes, fails.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1804_03479_b300 import inputs as I

pytestmark = pytest.mark.gpu

U_ROUND = 2.0 ** -53


@pytest.fixture(scope="module")
def M():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_03479_b300 import mhd
    mhd.lib()
    return mhd


def sum_bound(x):
    n = x.size
    return 2.0 * (n - 1) * U_ROUND * float(np.abs(x).sum())


def sine_faces(shape, seed):
    """B_d = a_d sin(2 pi m_d i_d / n_d + phase) on the faces: a non-zero
    discrete divergence of order one, different per axis."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    K, J, I_ = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    idx = (I_, J, K)
    B = np.empty((3, nz, ny, nx))
    for d in range(3):
        a, ph = rng.uniform(0.5, 2.0), rng.uniform(0, 2 * math.pi)
        B[d] = a * np.sin(2.0 * math.pi * (d + 1) * idx[d] / shape[d] + ph)
    return B


def poly_state(shape):
    nx, ny, nz = shape
    K, J, I_ = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    U = np.stack([(f + 1) * I_ + (f + 2) * J * J + (f + 3) * K + f for f in range(5)]).astype(float)
    B = np.stack([(d + 1) * I_ * J + K * K * (d + 2) - d for d in range(3)]).astype(float)
    return U, B


def dtype_of(prec):
    return np.float32 if prec == "fp32" else np.float64


def check_box(M, s, box, U, B, exact_sums=False):
    """U, B: the state the GPU holds (as doubles)."""
    m_g, r_g = s.divBs()
    m_o, r_o = orc.divB(B)
    assert m_g[box] == m_o, (box, m_g[box], m_o)
    bc2 = sum(((B[d] + np.roll(B[d], -1, axis=2 - d)) * 0.5) ** 2 for d in range(3))
    r_tol = sum_bound(bc2) / (2.0 * r_o * B[0].size) + 4 * U_ROUND * r_o
    assert abs(r_g[box] - r_o) <= r_tol, (box, r_g[box], r_o)
    sg = s.sums_boxes()[box]
    so = orc.sums(U, B)
    for f in range(8):
        x = U[f] if f < 5 else B[f - 5]
        if exact_sums:
            assert sg[f] == so[f], (box, f, sg[f], so[f])
        else:
            assert abs(sg[f] - so[f]) <= sum_bound(x), (box, f, sg[f], so[f])


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("shape", [(20, 12, 7), (33, 17, 9)])
def test_divB_and_sums_on_closed_form_fields(M, prec, shape):
    nx, ny, nz = shape
    st = I.uniform(0, shape=shape)
    dt = dtype_of(prec)
    B = sine_faces(shape, seed=nx).astype(dt)
    Up, Bp = poly_state(shape)
    s = M.Solver((nz, ny, nx), 1.0 / ny, st.gamma, "vl", "plm", "roe", prec, 0.3)
    try:
        s.set_state(st.U.astype(dt), B)
        Ug, Bg = s.get_state()          # what the GPU holds (MIXED keeps rho, M in FP32)
        check_box(M, s, 0, Ug.astype(np.float64), Bg.astype(np.float64))
        s.set_state(Up.astype(dt), Bp.astype(dt))
        check_box(M, s, 0, Up, Bp, exact_sums=True)
        m_o, _ = orc.divB(Bp)
        assert m_o > 1.0          # the polynomial field is far from divergence-free
    finally:
        s.free()


@pytest.mark.parametrize("integ,recon,solver", [("vl", "ppm", "hlld"), ("ctu", "plm", "roe")])
def test_divB_and_sums_on_a_stepped_abc_state(M, integ, recon, solver):
    st = I.abc(48, kmult=2, beta=0.5, seed=12, noise=1e-2)
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, integ, recon, solver, "fp64", 0.3)
    try:
        s.set_state(st.U, st.B)
        s.advance(3)
        U, B = s.get_state()
        check_box(M, s, 0, U, B)
        m, r = orc.divB(B)
        assert m / r <= 1e-13          # CT keeps div B at round-off
    finally:
        s.free()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_divB_and_sums_per_box_of_a_batch(M, prec):
    shapes = [(7, 12, 20), (9, 17, 33), (16, 16, 16)]    # (nz, ny, nx)
    dt = dtype_of(prec)
    s = M.Solver(None, 1.0 / 16, 5.0 / 3.0, "vl", "plm", "roe", prec, 0.3, shapes=shapes)
    try:
        states = []
        for b, sh in enumerate(shapes):
            nz, ny, nx = sh
            Up, Bp = poly_state((nx, ny, nz))
            Up = Up + 100.0 * b                   # each box its own sums
            s.set_state(Up.astype(dt), (sine_faces((nx, ny, nz), seed=b) if b == 1 else Bp).astype(dt), box=b)
            U, B = s.get_state(box=b)
            states.append((U.astype(np.float64), B.astype(np.float64)))
        for b in range(len(shapes)):
            check_box(M, s, b, *states[b], exact_sums=False)
    finally:
        s.free()
