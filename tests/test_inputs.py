"""Pins of the seeded initial conditions against closed forms.

ABC field (Eq. 20, Sec. 5.1 (v)) with face averages from the edge-averaged
potential A = B/k: every face value is the point value times sinc(k dx/2),
so the discrete magnetic energy is (A^2+B^2+C^2) L^3/2 sinc^2(k dx/2) and
the discrete edge curl is J = k_d sinc(k dx/2) B(edge) with
k_d = (2/dx) sin(k dx/2): the discrete form of J0 = 2 pi n B0 / L.
"""
import math

import numpy as np
import pytest

from paper_1804_03479_b300 import inputs as I


def divergence(B):
    return (np.roll(B[0], -1, 2) - B[0]) + (np.roll(B[1], -1, 1) - B[1]) + (np.roll(B[2], -1, 0) - B[2])


@pytest.mark.parametrize("maker", [
    lambda: I.abc(16, kmult=2, beta=0.5),
    lambda: I.linear_wave(16, "fast"),
    lambda: I.linear_wave(12, "alfven"),
    lambda: I.current_loop(32, 16, 8),
    lambda: I.orszag_tang(16, nz=4),
    lambda: I.abc_blasts(24, kmult=3, nblast=3, radius=0.12),
])
def test_initial_fields_are_divergence_free(maker):
    st = maker()
    assert np.abs(divergence(st.B)).max() < 1e-13 * np.abs(st.B).max()
    assert np.all(st.U[0] > 0)


@pytest.mark.parametrize("n,kmult", [(16, 1), (16, 2), (24, 3)])
def test_abc_discrete_energy_closed_form(n, kmult):
    st = I.abc(n, kmult=kmult, beta=1.0, noise=0.0)
    a = st.meta["A"]; k = st.meta["k"]; dx = st.dx
    s = math.sin(0.5 * k * dx) / (0.5 * k * dx)
    UB = 0.5 * (st.B ** 2).sum() * dx ** 3
    assert math.isclose(UB, 3 * a * a / 2 * s * s, rel_tol=1e-12)


def test_abc_discrete_current_closed_form():
    n, kmult = 16, 2
    st = I.abc(n, kmult=kmult, beta=1.0, noise=0.0)
    a = st.meta["A"]; k = st.meta["k"]; dx = st.dx
    Bx, By = st.B[0], st.B[1]
    # J_z on the z-edge (x_{i-1/2}, y_{j-1/2}) through cell k
    Jz = (By - np.roll(By, 1, 2)) / dx - (Bx - np.roll(Bx, 1, 1)) / dx
    xf = np.arange(n) * dx; yf = np.arange(n) * dx
    Y, X = np.meshgrid(yf, xf, indexing="ij")
    Bz_edge = a * np.sin(k * Y) + a * np.cos(k * X)
    kd = 2 / dx * math.sin(0.5 * k * dx)
    s = math.sin(0.5 * k * dx) / (0.5 * k * dx)
    assert np.allclose(Jz, kd * s * Bz_edge[None], atol=1e-12)
    # continuum limit: k_d s -> 2 pi n / L
    assert abs(kd * s - 2 * math.pi * kmult) / (2 * math.pi * kmult) < (k * dx) ** 2 / 4


def test_blast_energy_injection_exact():
    base = I.abc(24, kmult=3, beta=0.1, noise=1e-3, seed=2)
    st = I.abc_blasts(24, kmult=3, beta=0.1, nblast=4, E=1.0, radius=0.12, seed=2)
    dE = (st.U[4] - base.U[4]).sum() * st.dx ** 3
    assert math.isclose(dE, 4.0, rel_tol=1e-12)


def test_linear_wave_eigenvector_and_period():
    lam, r, bg = I.linear_wave_eigvec("fast")
    assert math.isclose(lam, 2.0, rel_tol=1e-12)
    lam, r, bg = I.linear_wave_eigvec("alfven")
    assert math.isclose(lam, 1.0, rel_tol=1e-12) and abs(r[0]) < 1e-12
    lam, r, bg = I.linear_wave_eigvec("slow")
    assert math.isclose(lam, 0.5, rel_tol=1e-12)
    st = I.linear_wave(8, "fast")
    assert math.isclose(st.meta["period"], 1 / math.sqrt(3) / 2.0, rel_tol=1e-12)
