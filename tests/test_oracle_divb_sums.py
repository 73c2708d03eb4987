"""Pins of the oracle's divergence (Eq. 16) and conserved sums (Sec. 5.1 (v))
against closed forms on fields where they are NOT zero.

The invariance tests elsewhere only see div B = 0 and unchanged sums; a
divergence that shifted the wrong way, summed instead of differencing,
dropped an axis or read the wrong stride, or a sum that skipped cells,
would pass them.  Here every expected value is a closed form:

- a face field B_d = sin(2 pi i_d / n_d) along one axis (face index i_d):
  the cell divergence is 2 sin(pi/n) cos(2 pi (i + 1/2)/n), whose largest
  magnitude (at i = 0) is sin(2 pi / n); the cell-centre field (mean of the
  two faces) is sin(2 pi (i + 1/2)/n) cos(pi/n), whose rms over the box is
  cos(pi/n)/sqrt(2);
- two axes superposed: the maxima add (both cosines peak at cell 0);
- a linear ramp B_x = i: divergence 1 per cell, except the periodic wrap
  cell (1 - n); along an outflow axis the face beyond the last cell is the
  last one, so the wrap cell's x-term is 0;
- a single unit face: divergence +-1 in its two cells, cell-centre field
  1/2 in both, rms sqrt(1/(2N));
- integer polynomial fields: sums by Faulhaber's formulas, exact in FP64.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc

SHAPE = (8, 12, 20)   # (nx, ny, nz): distinct sides, so an axis mix-up shows


def zero_field(shape=SHAPE):
    nx, ny, nz = shape
    return np.zeros((3, nz, ny, nx))


def face_index_grid(shape=SHAPE):
    nx, ny, nz = shape
    K, J, I_ = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return I_, J, K


@pytest.mark.parametrize("d", [0, 1, 2])
def test_divB_single_axis_sine(d):
    B = zero_field()
    idx = face_index_grid()[d]
    n = SHAPE[d]
    B[d] = np.sin(2.0 * math.pi * idx / n)
    m, r = orc.divB(B)
    assert abs(m - math.sin(2.0 * math.pi / n)) <= 1e-14
    assert abs(r - math.cos(math.pi / n) / math.sqrt(2.0)) <= 1e-14


@pytest.mark.parametrize("sy", [1.0, -1.0])
def test_divB_two_axes_add(sy):
    B = zero_field()
    I_, J, _ = face_index_grid()
    nx, ny, _ = SHAPE
    B[0] = np.sin(2.0 * math.pi * I_ / nx)
    B[1] = sy * np.sin(2.0 * math.pi * J / ny)
    m, r = orc.divB(B)
    assert abs(m - (math.sin(2.0 * math.pi / nx) + math.sin(2.0 * math.pi / ny))) <= 1e-14
    want_r = math.sqrt((math.cos(math.pi / nx) ** 2 + math.cos(math.pi / ny) ** 2) / 2.0)
    assert abs(r - want_r) <= 1e-14


def test_divB_ramp_periodic_and_outflow():
    nx = SHAPE[0]
    for d in range(3):
        B = zero_field()
        B[d] = face_index_grid()[d].astype(float)
        n = SHAPE[d]
        m, _ = orc.divB(B)
        assert m == n - 1                       # the wrap cell: 0 - (n - 1)
        m, _ = orc.divB(B, bc=1 << d)
        assert m == 1.0                         # outflow: the last cell's term is 0
        m, _ = orc.divB(B, bc=7 & ~(1 << d))   # outflow on the other axes only
        assert m == n - 1
    assert nx == 8


def test_divB_single_face_locality():
    nx, ny, nz = SHAPE
    N = nx * ny * nz
    for d in range(3):
        B = zero_field()
        B[d, 5, 7, 3] = 1.0
        m, r = orc.divB(B)
        assert m == 1.0
        assert abs(r - math.sqrt(0.5 / N)) <= 1e-16


def test_divB_of_a_gradient_field_is_its_laplacian():
    """B = grad(phi) on the faces, phi = cell values: the divergence is the
    7-point Laplacian, whose maximum for phi = delta at one cell is 6."""
    nx, ny, nz = SHAPE
    phi = np.zeros((nz, ny, nx))
    phi[4, 6, 2] = 1.0
    B = np.stack([phi - np.roll(phi, 1, axis=2), phi - np.roll(phi, 1, axis=1), phi - np.roll(phi, 1, axis=0)])
    m, _ = orc.divB(B)
    assert m == 6.0


def poly_state(shape=SHAPE):
    I_, J, K = face_index_grid(shape)
    U = np.stack([(f + 1) * I_ + (f + 2) * J * J + (f + 3) * K + f for f in range(5)]).astype(float)
    B = np.stack([(d + 1) * I_ * J + K * K * (d + 2) - d for d in range(3)]).astype(float)
    return U, B


def s1(n):      # sum_{i<n} i
    return n * (n - 1) // 2


def s2(n):      # sum_{i<n} i^2
    return (n - 1) * n * (2 * n - 1) // 6


def expected_poly_sums(shape=SHAPE):
    nx, ny, nz = shape
    N = nx * ny * nz
    out = []
    for f in range(5):
        out.append((f + 1) * s1(nx) * ny * nz + (f + 2) * s2(ny) * nx * nz + (f + 3) * s1(nz) * nx * ny + f * N)
    for d in range(3):
        out.append((d + 1) * s1(nx) * s1(ny) * nz + (d + 2) * s2(nz) * nx * ny - d * N)
    return out


def test_sums_closed_form_exact():
    U, B = poly_state()
    got = orc.sums(U, B)
    want = expected_poly_sums()
    assert len(got) == 8
    for f in range(8):
        assert got[f] == float(want[f]), (f, got[f], want[f])


def test_sums_see_every_cell():
    nx, ny, nz = SHAPE
    N = nx * ny * nz
    U = np.zeros((5, nz, ny, nx))
    B = np.zeros((3, nz, ny, nx))
    for f in range(5):
        U[f].flat[(37 * f + 11) % N] = 2.0 ** (f + 1)
        U[f].flat[N - 1] += 1.0                       # the last cell
        U[f].flat[0] += 0.5                           # the first cell
    for d in range(3):
        B[d].flat[N - 1 - d] = -3.0 * (d + 1)
    got = orc.sums(U, B)
    for f in range(5):
        assert got[f] == 2.0 ** (f + 1) + 1.5
    for d in range(3):
        assert got[5 + d] == -3.0 * (d + 1)
