"""Diagnostics on the GPU (mhd_energies: E_T, U_B, U_V and the |J|/|B|
refinement test of Sec. 4.3 / 4.5; mhd_helicity; mhd_pressure_gradient, the
refinement test of the blast run of Sec. 5.1) against the FP64 oracle, on
single boxes and a ragged batch, in FP64 and FP32."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1804_03479_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_03479_b300 import mhd
    mhd.lib()
    return mhd


def evolved(st, nsteps, scheme=("vl", "ppm", "hlld")):
    U, B = st.U.copy(), st.B.copy()
    for _ in range(nsteps):
        dt = orc.cfl_dt(U, B, st.dx, st.gamma, 0.3)
        orc.step(U, B, st.dx, st.gamma, dt, *scheme)
    return U, B


def check(g, o, tol):
    for k in ("E_T", "U_B", "U_V", "jb_max", "j_max"):
        assert abs(g[k] - o[k]) <= tol * abs(o[k]) + 1e-300, (k, g[k], o[k])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 3e-6)])
def test_energies_match_oracle(M, prec, tol):
    st = I.orszag_tang(32, nz=8)
    U, B = evolved(st, 3)
    s = M.Solver(U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", prec, 0.3)
    try:
        cast = np.float64 if prec == "fp64" else np.float32
        s.set_state(U.astype(cast), B.astype(cast))
        if prec == "fp32":
            U, B = U.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
        for thr in (0.05, 0.2, 1.0):
            o = orc.energies(U, B, st.dx, thr)
            g = s.energies(thr)
            check(g, o, tol)
            if prec == "fp64":
                assert g["n_above"] == o["n_above"], (thr, g["n_above"], o["n_above"])
            else:
                assert abs(g["n_above"] - o["n_above"]) <= max(2, 1e-3 * U[0].size)
    finally:
        s.free()


def test_energies_batch_ragged(M):
    boxes = [I.abc(16, kmult=1, beta=1.0, seed=31, noise=1e-2), I.orszag_tang(24, nz=5),
             I.abc(None, kmult=1, beta=0.5, seed=32, noise=3e-2, shape=(20, 12, 9))]
    s = M.Solver(None, None, 5 / 3, "vl", "plm", "roe", "fp64", 0.3,
                 shapes=[b.U.shape[1:] for b in boxes], dxs=[b.dx for b in boxes])
    try:
        for k, b in enumerate(boxes):
            s.set_state(b.U, b.B, box=k)
        got = s.energies_boxes(0.3)
        for k, b in enumerate(boxes):
            o = orc.energies(b.U, b.B, b.dx, 0.3)
            g = dict(E_T=got[k, 0], U_B=got[k, 1], U_V=got[k, 2], jb_max=got[k, 3], n_above=int(got[k, 4]),
                     j_max=got[k, 5])
            check(g, o, 1e-13)
            assert g["n_above"] == o["n_above"]
    finally:
        s.free()


def test_energy_conserved_and_magnetic_energy_decays_on_gpu(M):
    """E_T stays at round-off (finite volumes on a periodic box) while the
    unstable two-period ABC field (k = 4 pi) with its velocity noise loses a
    little magnetic energy to the flow and to numerical dissipation."""
    st = I.abc(32, kmult=2, beta=1.0, seed=5, noise=1e-2)
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", "fp64", 0.3)
    try:
        s.set_state(st.U, st.B)
        e0 = s.energies()
        s.advance(20)
        e1 = s.energies()
        assert abs(e1["E_T"] - e0["E_T"]) <= 1e-13 * e0["E_T"]
        assert e1["U_B"] < e0["U_B"]
    finally:
        s.free()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
def test_helicity_matches_oracle(M, prec):
    states = [I.abc(24, kmult=2, beta=1.0, seed=1, noise=0.0), I.abc_perturbed(16, kmult=2),
              I.orszag_tang(20, nz=6)]
    for st in states:
        s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", prec, 0.3)
        try:
            cast = np.float32 if prec == "fp32" else np.float64
            s.set_state(st.U.astype(cast), st.B.astype(cast))
            Bref = st.B.astype(cast).astype(np.float64)
            h = s.helicity()
            ho = orc.helicity(Bref, st.dx)
            assert abs(h - ho) <= 1e-10 * max(abs(ho), 1e-12), (st.meta.get("kind"), h, ho)
        finally:
            s.free()


def test_helicity_batch_ragged(M):
    boxes = [I.abc(16, kmult=1, beta=1.0, seed=31, noise=1e-2), I.abc_perturbed(12, kmult=2),
             I.abc(None, kmult=1, beta=0.5, seed=32, noise=3e-2, shape=(20, 12, 9))]
    s = M.Solver(None, None, 5 / 3, "vl", "plm", "roe", "fp64", 0.3,
                 shapes=[b.U.shape[1:] for b in boxes], dxs=[b.dx for b in boxes])
    try:
        for k, b in enumerate(boxes):
            s.set_state(b.U, b.B, box=k)
        h = s.helicities()
        for k, b in enumerate(boxes):
            ho = orc.helicity(b.B, b.dx)
            assert abs(h[k] - ho) <= 1e-10 * abs(ho), (k, h[k], ho)
        # the state is untouched: a step after the diagnostic equals a step without it
        U0, B0 = s.get_state(box=0)
        assert np.array_equal(U0, boxes[0].U)
    finally:
        s.free()


def blast_evolved(n=32, r0=0.1, nsteps=3):
    st = I.mhd_blast(n, r0=r0, density_noise=True)
    U, B = evolved(st, nsteps, ("vl", "plm", "roe"))
    return st, U, B


def check_pgrad(g, o, tol):
    assert abs(g["max"] - o["max"]) <= tol * o["max"], (g["max"], o["max"])
    assert g["counts"] == o["counts"], (g["counts"], o["counts"])


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
def test_pressure_gradient_matches_oracle(M, prec):
    """the indicator is computed in FP64 from the stored state on both sides,
    so the counts agree exactly and the maximum to rounding order"""
    st, U, B = blast_evolved()
    s = M.Solver(U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", prec, 0.3)
    try:
        if prec == "fp32":
            U, B = U.astype(np.float32), B.astype(np.float32)
        elif prec == "mixed":
            U = U.copy()
            U[:4] = U[:4].astype(np.float32)     # rho and M are stored in FP32
        s.set_state(U, B)
        Ur, Br = U.astype(np.float64), B.astype(np.float64)
        for scale, thr, nlev in [(10.0, 1.25, 4), (10.0, 40.0, 2), (0.5, 0.3, 1)]:
            o = orc.pressure_gradient(Ur, Br, st.dx, st.gamma, scale, thr, nlev)
            g = s.pressure_gradient(scale, thr, nlev)
            check_pgrad(g, o, 1e-12)
        assert o["counts"][0] > 0
    finally:
        s.free()


def test_pressure_gradient_batch_and_outflow(M):
    _, U1, B1 = blast_evolved(24, 0.12, 2)
    ob = I.open_box((20, 12, 9), seed=4)
    boxes = [(U1, B1, 1.0 / 24), (ob.U, ob.B, ob.dx)]
    s = M.Solver(None, None, 5 / 3, "vl", "plm", "roe", "fp64", 0.3,
                 shapes=[b[0].shape[1:] for b in boxes], dxs=[b[2] for b in boxes])
    try:
        for k, (U, B, dx) in enumerate(boxes):
            s.set_state(U, B, box=k)
        got = s.pressure_gradient_boxes(5.0, 0.5, 3)
        for k, (U, B, dx) in enumerate(boxes):
            o = orc.pressure_gradient(U, B, dx, 5 / 3, 5.0, 0.5, 3)
            check_pgrad(dict(max=got[k, 0], counts=[int(x) for x in got[k, 1:]]), o, 1e-12)
    finally:
        s.free()
    s = M.Solver(ob.U.shape[1:], ob.dx, ob.gamma, "vl", "plm", "roe", "fp64", 0.3)
    try:
        s.set_boundary(7)
        s.set_state(ob.U, ob.B)
        for bc in (7,):
            o = orc.pressure_gradient(ob.U, ob.B, ob.dx, ob.gamma, 2.0, 0.2, 3, bc=bc)
            check_pgrad(s.pressure_gradient(2.0, 0.2, 3), o, 1e-12)
    finally:
        s.free()


def test_pressure_gradient_leaves_the_step_unchanged(M):
    st, U, B = blast_evolved(24, 0.12, 1)
    out = []
    for call in (False, True):
        s = M.Solver(U.shape[1:], st.dx, st.gamma, "vl", "ppm", "hlld", "fp64", 0.3)
        try:
            s.set_state(U, B)
            s.advance(1)
            if call:
                s.pressure_gradient(10.0, 1.25)
            s.advance(1)
            out.append(s.get_state())
        finally:
            s.free()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_pressure_gradient_rejects_bad_arguments(M):
    st = I.uniform(8)
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", "fp64", 0.3)
    try:
        s.set_state(st.U, st.B)
        for args in [(0.0, 1.0, 1), (1.0, -1.0, 1), (1.0, 1.0, 0), (1.0, 1.0, 5)]:
            with pytest.raises(RuntimeError):
                s.pressure_gradient(*args)
            s.clear_error()                   # errors stay until cleared
        r = s.pressure_gradient(1.0, 0.0, 4)
        assert r["max"] < 1e-12 and r["counts"] == [0, 0, 0, 0]
    finally:
        s.free()
