"""Pins of the oracle's seven-wave eigensystem (the characteristic basis of
the reconstruction, Sec. 3.2 step 1) against numpy's eigensolver applied to
the quasi-linear form of Eqs. 1-4 in one dimension."""
import numpy as np
import pytest

from oracle import oracle as orc

GAMMA = 5.0 / 3.0


def jacobian(w, bn, gamma):
    """d w/dt + A d w/dx = 0 for w = (rho, v_n, v_t1, v_t2, P, B_t1, B_t2),
    B_n constant: the x-derivative terms of Eqs. 1-4 with P from Eq. 5."""
    rho, u, v, ww, P, b1, b2 = w
    A = np.zeros((7, 7))
    A[0, 0] = u; A[0, 1] = rho
    A[1, 1] = u; A[1, 4] = 1 / rho; A[1, 5] = b1 / rho; A[1, 6] = b2 / rho
    A[2, 2] = u; A[2, 5] = -bn / rho
    A[3, 3] = u; A[3, 6] = -bn / rho
    A[4, 1] = gamma * P; A[4, 4] = u
    A[5, 1] = b1; A[5, 2] = -bn; A[5, 5] = u
    A[6, 1] = b2; A[6, 3] = -bn; A[6, 6] = u
    return A


def random_states(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        w = np.array([rng.uniform(0.05, 5), *rng.normal(size=3), rng.uniform(0.01, 5), *rng.normal(size=2)])
        out.append((w, rng.normal()))
    # degenerate corners: B_t = 0, B_n = 0, a = c_a (triple umbilic), B = 0
    out.append((np.array([1.0, 0.3, 0.1, -0.2, 0.6, 0.0, 0.0]), 1.0))
    out.append((np.array([1.0, 0.3, 0.1, -0.2, 0.6, 0.5, -0.4]), 0.0))
    out.append((np.array([1.0, 0.0, 0.0, 0.0, 0.6, 0.0, 0.0]), np.sqrt(GAMMA * 0.6)))
    out.append((np.array([2.0, 0.1, 0.2, 0.3, 0.6, 0.0, 0.0]), 0.0))
    return out


@pytest.mark.parametrize("seed", [0, 1])
def test_eigen_decomposes_the_jacobian(seed):
    for w, bn in random_states(2000, seed):
        lam, R, L = orc.eigen(w, bn, GAMMA)
        A = jacobian(w, bn, GAMMA)
        scale = np.abs(A).max() + 1.0
        assert np.all(np.diff(lam) >= -1e-12 * scale)
        ev = np.sort(np.linalg.eigvals(A).real)
        assert np.allclose(ev, lam, atol=1e-6 * scale, rtol=0)
        # L R = I and A R = R diag(lam)
        assert np.abs(L @ R - np.eye(7)).max() < 1e-9 * (1 + np.abs(L).max() * np.abs(R).max())
        assert np.abs(A @ R - R * lam).max() < 1e-9 * scale * (1 + np.abs(R).max())


def test_eigenvalue_closed_forms():
    # rho = 1, P = 1/gamma (a = 1), B = (1, sqrt 2, 1/2): c_a = 1, c_f = 2, c_s = 1/2
    w = np.array([1.0, 0.25, 0.0, 0.0, 1 / GAMMA, np.sqrt(2.0), 0.5])
    lam, R, L = orc.eigen(w, 1.0, GAMMA)
    assert np.allclose(lam, 0.25 + np.array([-2, -1, -0.5, 0, 0.5, 1, 2]), atol=1e-14)
    # hydrodynamic limit: B = 0 -> sound speed a, all magnetic waves at v
    w = np.array([1.3, -0.4, 0.1, 0.2, 0.9, 0.0, 0.0])
    lam, R, L = orc.eigen(w, 0.0, GAMMA)
    a = np.sqrt(GAMMA * 0.9 / 1.3)
    assert np.allclose(lam, [-0.4 - a, -0.4, -0.4, -0.4, -0.4, -0.4, -0.4 + a], atol=1e-14)
