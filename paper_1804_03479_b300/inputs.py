"""Seeded synthetic initial conditions for the MHD patch advance.

This module is the one place both the CUDA path's callers and the oracle's
tests draw their inputs from.  It holds none of the scheme's arithmetic: it
only writes down initial states (numpy, float64) in the staggered layout

  U: (5, nz, ny, nx)  rho, Mx, My, Mz, e            (cell averages, Eq. 11)
  B: (3, nz, ny, nx)  Bx at x_{i-1/2}, By at y_{j-1/2}, Bz at z_{k-1/2}
                      (face averages, Eq. 14; no duplicated periodic face)

Face fields come from a vector potential averaged along cell edges, so that
Stokes' theorem makes them exact face averages with a discrete divergence
(Eq. 16) of zero to round-off.  Random numbers (velocity noise, blast sites)
come from numpy's PCG64 with an explicit seed.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class State:
    U: np.ndarray
    B: np.ndarray
    dx: float
    gamma: float
    meta: dict

    @property
    def shape(self):
        return self.U.shape[1:]


def _coords(nx, ny, nz, dx):
    """cell centres (Sec. 3.1: x_i = (i + 1/2) dx) and lower faces x_{i-1/2}."""
    xc = (np.arange(nx) + 0.5) * dx
    yc = (np.arange(ny) + 0.5) * dx
    zc = (np.arange(nz) + 0.5) * dx
    xf = np.arange(nx) * dx
    yf = np.arange(ny) * dx
    zf = np.arange(nz) * dx
    return xc, yc, zc, xf, yf, zf


def curl_edges(Ax, Ay, Az, dx):
    """Face averages of B = curl A from edge averages of A (Stokes).

    Edge storage: Ax[k,j,i] on the x-edge at (y_{j-1/2}, z_{k-1/2}) through
    cell column i; Ay[k,j,i] at (x_{i-1/2}, z_{k-1/2}); Az[k,j,i] at
    (x_{i-1/2}, y_{j-1/2}).  Periodic in all axes.
    """
    r = lambda a, ax: np.roll(a, -1, axis=ax)  # value at index + 1
    # axis order in arrays is (z, y, x)
    Bx = ((r(Az, 1) - Az) - (r(Ay, 0) - Ay)) / dx
    By = ((r(Ax, 0) - Ax) - (r(Az, 2) - Az)) / dx
    Bz = ((r(Ay, 2) - Ay) - (r(Ax, 1) - Ax)) / dx
    return np.stack([Bx, By, Bz])


def cell_centre_B(B):
    """mean of the two faces of each cell (the layout of Fig. 1)"""
    bx = 0.5 * (B[0] + np.roll(B[0], -1, axis=2))
    by = 0.5 * (B[1] + np.roll(B[1], -1, axis=1))
    bz = 0.5 * (B[2] + np.roll(B[2], -1, axis=0))
    return bx, by, bz


def conserved(rho, vx, vy, vz, P, B, gamma):
    """U from primitives with e from Eq. 5 and the face-mean cell-centre B."""
    bx, by, bz = cell_centre_B(B)
    e = P / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) + 0.5 * (bx * bx + by * by + bz * bz)
    return np.ascontiguousarray(np.stack([rho, rho * vx, rho * vy, rho * vz, e]).astype(np.float64))


def abc_potential(nx, ny, nz, dx, k, A, Bc, C):
    """Edge averages of the potential of the ABC field of Eq. 20.

    The field is an eigenfunction of curl (curl B = k B), so A_vec = B / k;
    each component is independent of its own coordinate, so its edge average
    is the value at the edge midpoint.
    """
    xc, yc, zc, xf, yf, zf = _coords(nx, ny, nz, dx)
    Z, Y, X = np.meshgrid(zf, yf, xc, indexing="ij")    # x-edges
    Ax = (A * np.sin(k * Z) + C * np.cos(k * Y)) / k
    Z, Y, X = np.meshgrid(zf, yc, xf, indexing="ij")    # y-edges
    Ay = (Bc * np.sin(k * X) + A * np.cos(k * Z)) / k
    Z, Y, X = np.meshgrid(zc, yf, xf, indexing="ij")    # z-edges
    Az = (C * np.sin(k * Y) + Bc * np.cos(k * X)) / k
    return Ax, Ay, Az


def abc(n, kmult=1, beta=1.0, gamma=5.0 / 3.0, noise=1e-3, seed=0, L=1.0, shape=None,
        A=None, rho0=1.0, drift=(0.0, 0.0, 0.0)):
    """Uniform plasma threaded by the ABC field (Eq. 20), k = 2 pi kmult / L.

    A = B = C (default 1/sqrt(3)); the gas pressure is P0 = beta * A^2 (the
    paper calls A = B = C = sqrt(P0) plasma beta 1).  The velocity is the
    uniform drift plus seeded Gaussian noise of rms noise * c_s per
    component, c_s = sqrt(gamma P0 / rho0).
    """
    nx, ny, nz = shape if shape is not None else (n, n, n)
    dx = L / ny if shape is not None else L / n
    a = 1.0 / math.sqrt(3.0) if A is None else A
    k = 2.0 * math.pi * kmult / L
    P0 = beta * a * a
    Ax, Ay, Az = abc_potential(nx, ny, nz, dx, k, a, a, a)
    B = curl_edges(Ax, Ay, Az, dx)
    cs = math.sqrt(gamma * P0 / rho0)
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((3, nz, ny, nx)) * (noise * cs)
    for d in range(3):
        v[d] += drift[d]
    rho = np.full((nz, ny, nx), rho0)
    P = np.full((nz, ny, nx), P0)
    U = conserved(rho, v[0], v[1], v[2], P, B, gamma)
    return State(U, np.ascontiguousarray(B), dx, gamma,
                 dict(kind="abc", k=k, A=a, P0=P0, beta=beta, seed=seed, noise=noise))


# Fourier modes of the unstable n = 1 perturbation of the ABC state (Eqs. 21-23):
# wave vector in units of 2 pi / L, then the cos and sin amplitude vectors
# (x, y, z components) in units of 1e-2 of the field amplitude.
ABC_EIGENMODE = (
    ((1, 1, 0), (2.37, -2.37, -3.23), (2.10, -2.10, 3.66)),
    ((1, 0, 1), (-3.48, -4.90, 3.48), (-3.18, 5.37, 3.18)),
    ((0, -1, 1), (-5.86, 3.60, 3.60), (5.60, 3.80, 3.80)),
    ((1, 0, -1), (2.08, -3.00, 2.08), (1.94, 3.22, 1.94)),
)


def _sinc(u):
    return np.where(np.abs(u) < 1e-300, 1.0, np.sin(u) / np.where(np.abs(u) < 1e-300, 1.0, u))


def abc_eigenmode_potential(nx, ny, nz, dx, amp, L=1.0):
    """Edge averages of a vector potential of the perturbation of Eqs. 21-23,
    scaled by amp (the paper's 1e-2 sqrt(P0) is amp = 1e-2 A at its beta = 1).

    Every mode a cos(k.x) + b sin(k.x) has k.a = k.b = 0, so it is the curl of
    (a x k) sin(k.x)/|k|^2 - (b x k) cos(k.x)/|k|^2.  The average of
    sin(k.x) along an edge of length dx in direction d is its midpoint value
    times sinc(k_d dx / 2).
    """
    xc, yc, zc, xf, yf, zf = _coords(nx, ny, nz, dx)
    pts = [np.meshgrid(zf, yf, xc, indexing="ij"),      # x-edges (z, y, x)
           np.meshgrid(zf, yc, xf, indexing="ij"),      # y-edges
           np.meshgrid(zc, yf, xf, indexing="ij")]      # z-edges
    A = [np.zeros((nz, ny, nx)) for _ in range(3)]
    for kv, a, b in ABC_EIGENMODE:
        k = 2.0 * math.pi / L * np.array(kv, dtype=float)
        k2 = float(k @ k)
        a = amp * 1e-2 * np.array(a)
        b = amp * 1e-2 * np.array(b)
        ca = np.cross(a, k) / k2
        cb = np.cross(b, k) / k2
        for d in range(3):
            Z, Y, X = pts[d]
            ph = k[0] * X + k[1] * Y + k[2] * Z
            w = float(_sinc(0.5 * k[d] * dx))
            A[d] += w * (ca[d] * np.sin(ph) - cb[d] * np.cos(ph))
    return A[0], A[1], A[2]


def abc_perturbed(n, kmult=2, beta=1.0, gamma=5.0 / 3.0, amp=None, drift=True, noise=0.0, seed=0, L=1.0):
    """The ABC relaxation run's initial state (Sec. 4.5): the n = kmult ABC
    field plus the perturbation of Eqs. 21-23 (amplitude 1e-2 of the field
    amplitude A by default), and a uniform drift along the box diagonal of
    magnitude c_s / (8 sqrt(gamma)) when drift is true."""
    a = 1.0 / math.sqrt(3.0)
    dx = L / n
    k = 2.0 * math.pi * kmult / L
    P0 = beta * a * a
    Ax, Ay, Az = abc_potential(n, n, n, dx, k, a, a, a)
    px, py, pz = abc_eigenmode_potential(n, n, n, dx, a if amp is None else amp, L)
    B = curl_edges(Ax + px, Ay + py, Az + pz, dx)
    cs = math.sqrt(gamma * P0)
    v0 = cs / (8.0 * math.sqrt(gamma)) / math.sqrt(3.0) if drift else 0.0
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((3, n, n, n)) * (noise * cs) + v0
    U = conserved(np.ones((n, n, n)), v[0], v[1], v[2], np.full((n, n, n), P0), B, gamma)
    return State(U, np.ascontiguousarray(B), dx, gamma,
                 dict(kind="abc_perturbed", k=k, A=a, P0=P0, beta=beta, drift=v0, seed=seed))


def _rotation_to_z(bhat):
    """rotation about the axis x + y = 0, z = 0 (direction (1, -1, 0)/sqrt 2)
    that takes the unit vector bhat (whose x-y projection lies along
    (1, 1, 0)) onto z"""
    u = np.array([1.0, -1.0, 0.0]) / math.sqrt(2.0)
    th = math.acos(max(-1.0, min(1.0, float(bhat[2]))))
    K = np.array([[0, -u[2], u[1]], [u[2], 0, -u[0]], [-u[1], u[0], 0]])
    best = None
    for ang in (th, -th):
        R = np.eye(3) + math.sin(ang) * K + (1.0 - math.cos(ang)) * (K @ K)
        err = float(np.abs(R @ bhat - np.array([0.0, 0.0, 1.0])).max())
        if best is None or err < best[0]:
            best = (err, R)
    return best[1]


def mhd_blast(n, r0=0.05, theta0=90.0, phi0=45.0, beta_amb=0.2, P_in=1.0, ratio=1e-2, rho0=1.0,
              gamma=5.0 / 3.0, density_noise=False, L=1.0):
    """Magnetised blast (Sec. 4.4): a static sphere of radius r0 at the box
    centre with pressure P_in in an ambient medium of pressure ratio * P_in,
    uniform density rho0, and a uniform field B0 along (cos phi0 sin theta0,
    sin phi0 sin theta0, cos theta0) with ambient beta = 2 P_amb / B0^2.
    With density_noise, the density inside 1.5 r0 carries the perturbation
    of Eq. 19 in coordinates rotated so that B is along z' (no pressure
    perturbation).  The paper takes r0, rho0, P and B0 from a reference it
    cites; these defaults keep its beta and its pressure contrast."""
    dx = L / n
    xc = (np.arange(n) + 0.5) * dx
    Z, Y, X = np.meshgrid(xc, xc, xc, indexing="ij")
    c = 0.5 * L
    dX, dY, dZ = X - c, Y - c, Z - c
    r = np.sqrt(dX * dX + dY * dY + dZ * dZ)
    P_amb = ratio * P_in
    B0 = math.sqrt(2.0 * P_amb / beta_amb)
    th, ph = math.radians(theta0), math.radians(phi0)
    bhat = np.array([math.cos(ph) * math.sin(th), math.sin(ph) * math.sin(th), math.cos(th)])
    rho = np.full((n, n, n), rho0)
    if density_noise:
        R = _rotation_to_z(bhat)
        xp = R[0, 0] * dX + R[0, 1] * dY + R[0, 2] * dZ
        yp = R[1, 0] * dX + R[1, 1] * dY + R[1, 2] * dZ
        tp = 2.0 * math.pi / r0
        d = (np.sin(tp / 0.08 * xp + math.pi / 4) + np.sin(tp / 0.10 * xp) + np.sin(tp / 0.12 * xp - math.pi / 4)
             + np.cos(tp / 0.08 * yp + math.pi / 4) + np.cos(tp / 0.10 * yp) + np.cos(tp / 0.12 * yp - math.pi / 4))
        rho = np.where(r < 1.5 * r0, rho0 * (1.0 + 2e-2 * d), rho)
    P = np.where(r < r0, P_in, P_amb)
    B = np.stack([np.full((n, n, n), B0 * bhat[d]) for d in range(3)])
    z = np.zeros((n, n, n))
    U = conserved(rho, z, z, z, P, B, gamma)
    return State(U, np.ascontiguousarray(B), dx, gamma,
                 dict(kind="mhd_blast", r0=r0, B0=B0, bhat=bhat, P_amb=P_amb, density_noise=density_noise))


# --- linear waves ----------------------------------------------------------

WAVES = {"fast": 6, "alfven": 5, "slow": 4, "entropy": 3}


def linear_wave_eigvec(wave, gamma=5.0 / 3.0):
    """Right eigenvector of the 1-D primitive MHD system at the background.

    Background in the wave frame: rho = 1, P = 1/gamma, v = 0,
    B = (B_n, B_t1, B_t2) = (1, sqrt 2, 1/2), so a = 1, c_a = 1, c_f = 2,
    c_s = 1/2.  The quasi-linear matrix of Eqs. 1-4 in the variables
    (rho, v_n, v_t1, v_t2, P, B_t1, B_t2) is diagonalised with numpy; the
    eigenvector is normalised to unit length with a positive leading entry.
    Returns (eigenvalue, eigenvector, background dict).
    """
    rho, P, bn, b1, b2 = 1.0, 1.0 / gamma, 1.0, math.sqrt(2.0), 0.5
    Am = np.zeros((7, 7))
    Am[0, 1] = rho
    Am[1, 4] = 1.0 / rho; Am[1, 5] = b1 / rho; Am[1, 6] = b2 / rho
    Am[2, 5] = -bn / rho
    Am[3, 6] = -bn / rho
    Am[4, 1] = gamma * P
    Am[5, 1] = b1; Am[5, 2] = -bn
    Am[6, 1] = b2; Am[6, 3] = -bn
    lam, vec = np.linalg.eig(Am)
    order = np.argsort(lam.real)
    lam = lam.real[order]; vec = vec.real[:, order]
    idx = WAVES[wave]
    r = vec[:, idx] / np.linalg.norm(vec[:, idx])
    lead = r[np.argmax(np.abs(r) > 1e-12)]
    if lead < 0:
        r = -r
    return lam[idx], r, dict(rho=rho, P=P, bn=bn, b1=b1, b2=b2)


def _edge_avg_sin(kv, x0, dx):
    """(1/dx) int_{x0-dx/2}^{x0+dx/2} of exp(i k x) -> factor sinc(k dx / 2)."""
    u = 0.5 * kv * dx
    return np.sinc(u / np.pi)  # numpy sinc is sin(pi x)/(pi x)


def linear_wave(n, wave="fast", amp=1e-6, gamma=5.0 / 3.0, L=1.0, shape=None, direction=(1, 1, 1)):
    """Travelling linear MHD wave along the box diagonal (Sec. 5.1 (i)).

    Wave vector k = 2 pi (1, 1, 1) / L in a cube (one period per box length
    along each axis).  Cell quantities are point values at the centres; the
    perturbation of B comes from the edge-averaged potential
    A = (dB x k) / |k|^2 sin(k.x), the uniform background B on the faces.
    """
    nx, ny, nz = shape if shape is not None else (n, n, n)
    dx = L / nx
    lam, r, bg = linear_wave_eigvec(wave, gamma)
    d = np.asarray(direction, dtype=float)
    kvec = 2.0 * math.pi * d / L
    nhat = d / np.linalg.norm(d)
    # transverse basis: t1 perpendicular to n in the plane with z, t2 = n x t1
    t1 = np.cross(nhat, [0.0, 0.0, 1.0]) if abs(nhat[2]) < 0.9 else np.cross(nhat, [1.0, 0.0, 0.0])
    t1 = -t1 / np.linalg.norm(t1)
    t2 = np.cross(nhat, t1)
    B0 = bg["bn"] * nhat + bg["b1"] * t1 + bg["b2"] * t2
    dv = amp * (r[1] * nhat + r[2] * t1 + r[3] * t2)
    dB = amp * (r[5] * t1 + r[6] * t2)
    avec = np.cross(dB, kvec) / (kvec @ kvec)
    xc, yc, zc, xf, yf, zf = _coords(nx, ny, nz, dx)
    sx = _edge_avg_sin(kvec[0], 0, dx); sy = _edge_avg_sin(kvec[1], 0, dx); sz = _edge_avg_sin(kvec[2], 0, dx)

    def phase(X, Y, Z):
        return kvec[0] * X + kvec[1] * Y + kvec[2] * Z

    Z, Y, X = np.meshgrid(zf, yf, xc, indexing="ij")
    Ax = avec[0] * np.sin(phase(X, Y, Z)) * sx
    Z, Y, X = np.meshgrid(zf, yc, xf, indexing="ij")
    Ay = avec[1] * np.sin(phase(X, Y, Z)) * sy
    Z, Y, X = np.meshgrid(zc, yf, xf, indexing="ij")
    Az = avec[2] * np.sin(phase(X, Y, Z)) * sz
    B = curl_edges(Ax, Ay, Az, dx)
    for m in range(3):
        B[m] += B0[m]
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    c = np.cos(phase(X, Y, Z))
    rho = bg["rho"] + amp * r[0] * c
    P = bg["P"] + amp * r[4] * c
    vx = dv[0] * c; vy = dv[1] * c; vz = dv[2] * c
    U = conserved(rho, vx, vy, vz, P, B, gamma)
    speed = lam  # background at rest
    period = (L / np.linalg.norm(d)) / abs(speed) if speed != 0 else float("inf")
    return State(U, np.ascontiguousarray(B), dx, gamma,
                 dict(kind="linear_wave", wave=wave, amp=amp, speed=speed, period=period))


def current_loop(nx=512, ny=256, nz=256, beta=1e-3, gamma=5.0 / 3.0, amp=1e-3, R0=0.3,
                 centre=(1.0, 0.5), vel=(2.0, 2.0, 2.0), noise=0.0, seed=0):
    """Low-beta ABC background (k = 2 pi) plus an advected current loop.

    Box 2 x 1 x 1 with dx = 1/ny.  The loop adds A_z = amp (R0 - r) for
    r < R0 (r the distance from the loop axis in the x-y plane, periodic),
    so B gains a field of magnitude amp inside the loop.  Uniform rho = 1,
    P0 = beta A^2 with A = 1/sqrt(3), bulk velocity vel.
    """
    dx = 1.0 / ny
    a = 1.0 / math.sqrt(3.0)
    k = 2.0 * math.pi
    Ax, Ay, Az = abc_potential(nx, ny, nz, dx, k, a, a, a)
    xc, yc, zc, xf, yf, zf = _coords(nx, ny, nz, dx)
    Lx, Ly = nx * dx, ny * dx
    Z, Y, X = np.meshgrid(zc, yf, xf, indexing="ij")
    ddx = (X - centre[0] + 0.5 * Lx) % Lx - 0.5 * Lx
    ddy = (Y - centre[1] + 0.5 * Ly) % Ly - 0.5 * Ly
    r = np.sqrt(ddx * ddx + ddy * ddy)
    Az = Az + np.where(r < R0, amp * (R0 - r), 0.0)
    B = curl_edges(Ax, Ay, Az, dx)
    P0 = beta * a * a
    rng = np.random.default_rng(seed)
    shp = (nz, ny, nx)
    v = [np.full(shp, vel[d]) for d in range(3)]
    if noise > 0:
        cs = math.sqrt(gamma * P0)
        for d in range(3):
            v[d] = v[d] + rng.standard_normal(shp) * noise * cs
    U = conserved(np.ones(shp), v[0], v[1], v[2], np.full(shp, P0), B, gamma)
    return State(U, np.ascontiguousarray(B), dx, gamma, dict(kind="current_loop", beta=beta, P0=P0))


def abc_blasts(n=384, kmult=3, beta=0.1, nblast=10, E=1.0, radius=0.05, gamma=5.0 / 3.0, seed=2,
               noise=1e-3):
    """ABC field (Eq. 20) at k = 2 pi kmult plus seeded Sedov-type blasts.

    Sites uniform in the unit box (PCG64, seed).  Each blast adds the
    pressure (gamma-1) E / V to the cells whose centres lie within `radius`
    (periodic distance), V being the summed volume of those cells, so the
    injected thermal energy is exactly E per site.
    """
    st = abc(n, kmult=kmult, beta=beta, gamma=gamma, noise=noise, seed=seed)
    dx = st.dx
    rng = np.random.default_rng(seed + 1000)
    sites = rng.uniform(0.0, 1.0, size=(nblast, 3))
    W_P = np.zeros((n, n, n))
    m = int(np.ceil(radius / dx)) + 1
    for s in sites:
        # cells of the periodic cube around the site; their centre offsets
        idx = [np.arange(int(np.floor(c / dx)) - m, int(np.floor(c / dx)) + m + 1) for c in s]
        off = [((ix + 0.5) * dx - c + 0.5) % 1.0 - 0.5 for ix, c in zip(idx, s)]
        d2 = off[2][:, None, None] ** 2 + off[1][None, :, None] ** 2 + off[0][None, None, :] ** 2
        mask = d2 < radius * radius
        vol = mask.sum() * dx ** 3
        if vol > 0:
            kk, jj, ii = np.nonzero(mask)
            np.add.at(W_P, (idx[2][kk] % n, idx[1][jj] % n, idx[0][ii] % n), (gamma - 1.0) * E / vol)
    # add to the total energy: e += dP / (gamma - 1)
    st.U[4] += W_P / (gamma - 1.0)
    st.meta.update(kind="abc_blasts", sites=sites.tolist(), E=E, radius=radius)
    return st


def orszag_tang(n, nz=None, gamma=5.0 / 3.0, L=1.0):
    """Orszag-Tang vortex (Eq. 18) extruded along z.

    rho0 = 25/(36 pi), P0 = 5/(12 pi) (C_s = 1, sqrt(P0/gamma) = 1/sqrt(4 pi));
    B from A_z = sqrt(P0/gamma) (cos(2 pi y)/(2 pi) + cos(4 pi x)/(4 pi)) L.
    """
    nz = n if nz is None else nz
    dx = L / n
    rho0 = 25.0 / (36.0 * math.pi)
    P0 = 5.0 / (12.0 * math.pi)
    cs = math.sqrt(gamma * P0 / rho0)
    b0 = math.sqrt(P0 / gamma)
    xc, yc, zc, xf, yf, zf = _coords(n, n, nz, dx)
    kk = 2.0 * math.pi / L
    Ax = np.zeros((nz, n, n)); Ay = np.zeros((nz, n, n))
    Z, Y, X = np.meshgrid(zc, yf, xf, indexing="ij")
    Az = b0 * (np.cos(kk * Y) / kk + np.cos(2 * kk * X) / (2 * kk))
    B = curl_edges(Ax, Ay, Az, dx)
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    vx = -cs * np.sin(kk * Y)
    vy = cs * np.sin(kk * X)
    shp = (nz, n, n)
    U = conserved(np.full(shp, rho0), vx, vy, np.zeros(shp), np.full(shp, P0), B, gamma)
    return State(U, np.ascontiguousarray(B), dx, gamma, dict(kind="orszag_tang"))


def uniform(n, rho=1.0, v=(0.3, -0.2, 0.1), P=0.7, Bv=(0.4, -0.5, 0.6), gamma=5.0 / 3.0, shape=None):
    nx, ny, nz = shape if shape is not None else (n, n, n)
    shp = (nz, ny, nx)
    B = np.stack([np.full(shp, Bv[m]) for m in range(3)])
    U = conserved(np.full(shp, rho), np.full(shp, v[0]), np.full(shp, v[1]), np.full(shp, v[2]),
                  np.full(shp, P), B, gamma)
    return State(U, np.ascontiguousarray(B), 1.0 / nx, gamma, dict(kind="uniform"))


def open_box(shape, seed=0, gamma=5.0 / 3.0):
    """Smooth state for boxes with outflow (zero-gradient) sides: each field
    component depends only on the two other coordinates (B_x(y, z), B_y(z, x),
    B_z(x, y)), so the face fields are divergence-free under any mix of
    periodic and outflow sides, whatever the box lengths; density, velocity
    and pressure carry a smooth part plus 5 % (pressure 10 %) uniform noise,
    with pressure near 0.5 (beta of order one)."""
    nx, ny, nz = shape
    dx = 1.0 / max(shape)
    rng = np.random.default_rng(seed)
    xc, yc, zc, _, _, _ = _coords(nx, ny, nz, dx)
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    ph = rng.uniform(0.0, 2.0 * np.pi, 10)
    tp = 2.0 * np.pi
    B = np.stack([0.5 + 0.2 * np.sin(tp * Y + ph[0]) * np.cos(tp * Z + ph[1]),
                  0.3 + 0.2 * np.sin(tp * Z + ph[2]) * np.cos(tp * X + ph[3]),
                  -0.2 + 0.2 * np.sin(tp * X + ph[4]) * np.cos(tp * Y + ph[5])])
    rho = 1.0 + 0.2 * np.sin(tp * (X + Y) + ph[6]) + 0.05 * rng.uniform(-1.0, 1.0, X.shape)
    v = [0.3 * np.sin(tp * (Y + Z) + ph[7 + m]) + 0.05 * rng.uniform(-1.0, 1.0, X.shape) for m in range(3)]
    P = 0.5 + 0.05 * rng.uniform(-1.0, 1.0, X.shape)
    U = conserved(rho, v[0], v[1], v[2], P, B, gamma)
    return State(U, np.ascontiguousarray(B), dx, gamma, dict(kind="open_box"))


def shock_tube(wl, wr, bn, n, axis=0, m=2, L=2.0, gamma=5.0 / 3.0):
    """1-D Riemann problem (Sec. 5.1 (ii), Table 1 states) on a periodic line
    of length L along `axis`, with m cells across: the left state fills
    [L/4, 3L/4) and the right state the rest, so the problem itself sits at
    3L/4 and its mirror image at L/4; both fans stay apart while their speeds
    times t are below L/4.  wl, wr = (rho, v_n, v_t1, v_t2, P, B_t1, B_t2) in
    the frame of `axis` (t1 = axis+1, t2 = axis+2 cyclic), bn the uniform
    normal field.  Face fields are the (piecewise constant) cell values."""
    dx = L / n
    shp = [m, m, m]
    shp[2 - axis] = n                        # array order (z, y, x)
    line = (np.arange(n) + 0.5) * dx
    left = (line >= 0.25 * L) & (line < 0.75 * L)
    wl, wr = np.asarray(wl, float), np.asarray(wr, float)
    prof = np.where(left[None, :], wl[:, None], wr[:, None])     # (7, n)
    bshape = [1, 1, 1]
    bshape[2 - axis] = n
    def field(v):
        return np.broadcast_to(v.reshape(bshape), shp).copy()
    t1, t2 = (axis + 1) % 3, (axis + 2) % 3
    vel = [None] * 3
    vel[axis], vel[t1], vel[t2] = field(prof[1]), field(prof[2]), field(prof[3])
    Bc = [None] * 3
    Bc[axis] = np.full(shp, float(bn))
    Bc[t1], Bc[t2] = field(prof[5]), field(prof[6])
    B = np.stack(Bc)
    U = conserved(field(prof[0]), vel[0], vel[1], vel[2], field(prof[4]), B, gamma)
    return State(U, np.ascontiguousarray(B), dx, gamma, dict(kind="shock_tube", axis=axis, L=L))


def box_sides(nbox=48, seed=1, choices=(32, 48, 64, 96, 128, 192)):
    """Side lengths of the batched uneven workload: uniform over `choices`."""
    rng = np.random.default_rng(seed)
    return [int(s) for s in rng.choice(np.asarray(choices), size=nbox)]


def batch_box(i, side, seed=1):
    """Initial state of box i of the batched workload: linear fast, Alfven or
    slow waves (amplitude 1e-6) and ABC fields at k = 2 pi or 4 pi, in turn."""
    kind = i % 5
    if kind == 0:
        return linear_wave(side, "fast")
    if kind == 1:
        return linear_wave(side, "alfven")
    if kind == 2:
        return linear_wave(side, "slow")
    if kind == 3:
        return abc(side, kmult=1, beta=1.0, seed=seed * 1000 + i)
    return abc(side, kmult=2, beta=0.5, seed=seed * 1000 + i)
