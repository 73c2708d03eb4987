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


def test_abc_eigenmode_perturbation_matches_eqs_21_23():
    """face averages of the perturbation (Eqs. 21-23) against a midpoint-rule
    quadrature of the printed Fourier modes over a few faces, and a discrete
    divergence at round-off"""
    n = 16
    amp = 0.4
    st0 = I.abc(n, kmult=2, beta=1.0, noise=0.0)
    st = I.abc_perturbed(n, kmult=2, beta=1.0, amp=amp, drift=False)
    dB = st.B - st0.B
    dx = st.dx

    def point(x, y, z):
        out = np.zeros(3)
        for kv, a, b in I.ABC_EIGENMODE:
            ph = 2 * np.pi * (kv[0] * x + kv[1] * y + kv[2] * z)
            out += 1e-2 * amp * (np.array(a) * np.cos(ph) + np.array(b) * np.sin(ph))
        return out

    q = (np.arange(40) + 0.5) / 40
    rng = np.random.default_rng(0)
    for _ in range(6):
        i, j, k = rng.integers(0, n, 3)
        # Bx face at x_{i-1/2}, averaged over y, z
        v = np.mean([point(i * dx, (j + a) * dx, (k + b) * dx)[0] for a in q for b in q])
        assert abs(dB[0, k, j, i] - v) <= 1e-5 * amp
        v = np.mean([point((i + a) * dx, j * dx, (k + b) * dx)[1] for a in q for b in q])
        assert abs(dB[1, k, j, i] - v) <= 1e-5 * amp
        v = np.mean([point((i + a) * dx, (j + b) * dx, k * dx)[2] for a in q for b in q])
        assert abs(dB[2, k, j, i] - v) <= 1e-5 * amp
    div = (np.roll(st.B[0], -1, 2) - st.B[0]) + (np.roll(st.B[1], -1, 1) - st.B[1]) + (np.roll(st.B[2], -1, 0) - st.B[2])
    assert np.abs(div).max() <= 1e-14


def test_eigenmode_amplitude_vectors_are_transverse():
    for kv, a, b in I.ABC_EIGENMODE:
        assert abs(np.dot(kv, a)) < 1e-12 and abs(np.dot(kv, b)) < 1e-12


def test_abc_perturbed_drift():
    st = I.abc_perturbed(8, kmult=2, beta=1.0)
    v = st.U[1:4] / st.U[0]
    cs = np.sqrt(st.gamma * st.meta["P0"])
    mag = np.sqrt((v ** 2).sum(axis=0))
    assert np.allclose(mag, cs / (8 * np.sqrt(st.gamma)), rtol=1e-12)
    assert np.allclose(v[0], v[1]) and np.allclose(v[1], v[2])


@pytest.mark.parametrize("theta0", [90.0, 35.26438968, 85.0])
def test_mhd_blast(theta0):
    n = 32
    st = I.mhd_blast(n, r0=0.1, theta0=theta0, phi0=45.0, density_noise=True)
    W_P = (st.gamma - 1) * (st.U[4] - 0.5 * (st.U[1] ** 2 + st.U[2] ** 2 + st.U[3] ** 2) / st.U[0]
                            - 0.5 * (st.B ** 2).sum(axis=0))
    assert np.isclose(W_P.max(), 1.0) and np.isclose(W_P.min(), 1e-2)
    B0 = st.meta["B0"]
    assert np.isclose(2 * 1e-2 / B0 ** 2, 0.2)
    bh = st.B[:, 0, 0, 0] / B0
    assert np.allclose(bh, st.meta["bhat"])
    # the rotation maps the field direction onto z' and preserves lengths
    R = I._rotation_to_z(st.meta["bhat"])
    assert np.allclose(R @ st.meta["bhat"], [0, 0, 1], atol=1e-12)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-12)
    # density perturbation: only inside 1.5 r0, of at most 6 x 2e-2
    rho = st.U[0]
    c = (np.arange(n) + 0.5) / n - 0.5
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    assert np.all(rho[r >= 0.15] == 1.0)
    assert np.abs(rho - 1.0).max() <= 0.12 + 1e-12
    assert np.abs(rho[r < 0.15] - 1.0).max() > 1e-3


def test_open_box_divergence_free_under_any_boundary_mix():
    """each component is independent of its own coordinate, so the face
    differences along its axis vanish whether that side wraps or not"""
    st = I.open_box((24, 20, 18), seed=3)
    B = st.B
    assert np.abs(np.diff(B[0], axis=2)).max() < 1e-15
    assert np.abs(np.diff(B[1], axis=1)).max() < 1e-15
    assert np.abs(np.diff(B[2], axis=0)).max() < 1e-15
    assert np.abs(divergence(B)).max() < 1e-15
    assert np.all(st.U[0] > 0.7)
    assert st.U.shape == (5, 18, 20, 24) and abs(st.dx - 1.0 / 24) < 1e-16
