"""GPU (libmhd.so, sm_103a) against the FP64 CPU oracle, through the C ABI.

FP64 bar: relative L1 per field, sum|gpu - oracle| / sum|oracle|, at most
1e-12 after one step from bitwise-identical input, repeated for 10 steps with
the GPU re-seeded from the oracle state before each step.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1804_03479_b300 import inputs as I

pytestmark = pytest.mark.gpu

COMBOS = [(i, r, s) for i in ("vl", "ctu") for r in ("plm", "ppm") for s in ("roe", "hlld", "hlle")]
COMBOS_ALL = COMBOS + [("vl", "plm_prim", "hlle"), ("vl", "plm_prim", "roe")]
TOL64 = 1e-12


@pytest.fixture(scope="module")
def M():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_03479_b300 import mhd
    mhd.lib()
    return mhd


def rel_l1(a, b):
    den = np.abs(b).sum()
    return np.abs(a - b).sum() / (den if den > 0 else 1.0)


def assert_state_close(Ug, Bg, U, B, tol, what="", mfloor=0.0):
    """relative L1 per field; mfloor > 0 puts a floor of mfloor * sum(rho)
    under the momentum denominators (for fields that are themselves a tiny
    perturbation of an O(1) background, e.g. a 1e-6 linear wave)"""
    for f in range(5):
        if f in (1, 2, 3) and mfloor > 0:
            den = max(np.abs(U[f]).sum(), mfloor * np.abs(U[0]).sum())
            r = np.abs(Ug[f] - U[f]).sum() / den
        else:
            r = rel_l1(Ug[f], U[f])
        assert r <= tol, f"{what} U[{f}] rel L1 {r:.3e}"
    for d in range(3):
        r = rel_l1(Bg[d], B[d])
        assert r <= tol, f"{what} B[{d}] rel L1 {r:.3e}"


def run_parity(M, st, integ, recon, solver, nsteps, tol=TOL64, mfloor=0.0):
    U, B = st.U.copy(), st.B.copy()
    s = M.Solver(U.shape[1:], st.dx, st.gamma, integ, recon, solver, "fp64", 0.3)
    try:
        for it in range(nsteps):
            s.set_state(U, B)
            dt = orc.cfl_dt(U, B, st.dx, st.gamma, 0.3)
            dtg = s.cfl_dt()
            assert abs(dtg - dt) <= 1e-14 * dt
            s.step(dt)
            orc.step(U, B, st.dx, st.gamma, dt, integ, recon, solver)
            Ug, Bg = s.get_state()
            assert_state_close(Ug, Bg, U, B, tol, f"{integ}/{recon}/{solver} step {it + 1}", mfloor)
    finally:
        s.free()


@pytest.mark.parametrize("integ,recon,solver", COMBOS_ALL)
def test_fp64_parity_abc32(M, integ, recon, solver):
    """32^3 ABC, k = 2 pi, beta = 1, noise 1e-3 c_s, seed 0; 10 steps at CFL 0.3."""
    st = I.abc(32, kmult=1, beta=1.0, seed=0)
    run_parity(M, st, integ, recon, solver, 10)


@pytest.mark.parametrize("integ,recon,solver", [("vl", "plm", "roe"), ("ctu", "ppm", "hlld"),
                                                ("vl", "ppm", "hlle"), ("ctu", "plm", "roe")])
def test_fp64_parity_ragged(M, integ, recon, solver):
    """non-cubic box whose sides are not multiples of the 32 x 8 tiles"""
    st = I.abc(None, kmult=1, beta=0.5, seed=5, noise=3e-2, shape=(40, 24, 20))
    run_parity(M, st, integ, recon, solver, 3)


@pytest.mark.parametrize("shape", [(1, 16, 16), (16, 1, 8), (9, 7, 1), (33, 9, 9)])
def test_fp64_parity_thin_boxes(M, shape):
    # dx = 1/16 and k = 2 pi whatever the shape (abc() takes dx = L / ny and
    # k = 2 pi kmult / L for a given shape)
    L = shape[1] / 16.0
    st = I.abc(None, kmult=L, beta=0.5, seed=6, noise=5e-2, shape=shape, L=L)
    run_parity(M, st, "vl", "ppm", "roe", 2)
    run_parity(M, st, "ctu", "plm", "hlld", 2)


@pytest.mark.parametrize("integ,recon,solver", [("vl", "plm", "roe"), ("ctu", "ppm", "hlld"),
                                                ("vl", "ppm", "hlld"), ("ctu", "plm", "roe")])
def test_fp64_parity_abc64_config(M, integ, recon, solver):
    """the 256^3 workload's initial condition (k = 4 pi, beta = 0.5) at 64^3"""
    st = I.abc(64, kmult=2, beta=0.5, seed=0)
    run_parity(M, st, integ, recon, solver, 3)


def test_fp64_parity_linear_wave(M):
    """amplitude 1e-6 on rho = 1, P = 3/5, |B| ~ 1.6: the momentum is itself
    a 1e-6 perturbation, so its denominator is floored at 1e-2 sum(rho)
    (rounding of the O(1) flux terms is ~1e-16 per cell)"""
    st = I.linear_wave(32, "fast")
    run_parity(M, st, "ctu", "plm", "roe", 3, mfloor=1e-2)
    st = I.linear_wave(32, "slow")
    run_parity(M, st, "vl", "ppm", "hlld", 3, mfloor=1e-2)


CONFIG2 = [(i, r, s) for i in ("vl", "ctu") for r in ("plm", "ppm") for s in ("roe", "hlld")]
# stated per-field bound on the FP32 path's relative L1 against the FP64
# oracle after 10 steps of the 256^3 workload's initial state at 64^3
# (rho, Mx, My, Mz, e, Bx, By, Bz); the momentum is the 1e-3 c_s noise plus
# what the ABC field drives, a small denominator
FP32_TOL64 = np.array([3e-6, 1e-3, 1e-3, 1e-3, 3e-6, 3e-6, 3e-6, 3e-6])


@pytest.mark.parametrize("integ,recon,solver", CONFIG2)
def test_fp32_error_statement_config2_64(M, integ, recon, solver):
    """The eight FP32 schemes of the 256^3 workload ({VL, CTU} x {PLM, PPM} x
    {Roe, HLLD}) on its initial state (k = 4 pi, beta = 0.5, seed 0) at 64^3:
    10 steps with the oracle's dt, relative L1 per field against the FP64
    oracle within FP32_TOL64."""
    st = I.abc(64, kmult=2, beta=0.5, seed=0)
    U, B = st.U.copy(), st.B.copy()
    s = M.Solver(U.shape[1:], st.dx, st.gamma, integ, recon, solver, "fp32", 0.3)
    try:
        s.set_state(U.astype(np.float32), B.astype(np.float32))
        for _ in range(10):
            dt = orc.cfl_dt(U, B, st.dx, st.gamma, 0.3)
            s.step(dt)
            orc.step(U, B, st.dx, st.gamma, dt, integ, recon, solver)
        Ug, Bg = s.get_state()
        errs = np.array([rel_l1(Ug[f].astype(np.float64), U[f]) for f in range(5)] +
                        [rel_l1(Bg[d].astype(np.float64), B[d]) for d in range(3)])
        print("fp32-l1", integ, recon, solver, " ".join("%.2e" % e for e in errs))
        assert np.all(errs <= FP32_TOL64), errs
    finally:
        s.free()


def neighbourhood(U, B, k, j, i, r):
    idx = lambda c, n: np.arange(c - r, c + r + 1) % n
    nz, ny, nx = U.shape[1:]
    kk, jj, ii = idx(k, nz), idx(j, ny), idx(i, nx)
    sub = np.ix_(kk, jj, ii)
    return (np.ascontiguousarray(np.stack([U[f][sub] for f in range(5)])),
            np.ascontiguousarray(np.stack([B[d][sub] for d in range(3)])))


@pytest.mark.parametrize("integ,recon,solver,prec,tol", [
    ("vl", "plm", "roe", "fp64", TOL64),
    ("ctu", "ppm", "hlld", "fp64", TOL64),
    ("vl", "plm", "roe", "fp32", 1e-6),
])
def test_full_size_sampled(M, integ, recon, solver, prec, tol):
    """256^3 (the benchmark workload, same launch configuration): one GPU step
    with the device CFL dt, then 24 sampled cells recomputed by the oracle
    on 21^3 periodic neighbourhoods (the step's dependency radius is < 10)."""
    st = I.abc(256, kmult=2, beta=0.5, seed=0)
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, integ, recon, solver, prec, 0.3)
    try:
        dt_cast = np.float32 if prec == "fp32" else np.float64
        U0 = st.U.astype(dt_cast)
        B0 = st.B.astype(dt_cast)
        s.set_state(U0, B0)
        s.advance(1)
        dt = s.last_dt()
        Ug, Bg = s.get_state()
    finally:
        s.free()
    U0d, B0d = U0.astype(np.float64), B0.astype(np.float64)
    dto = orc.cfl_dt(U0d, B0d, st.dx, st.gamma, 0.3)
    assert abs(dt - dto) <= (1e-14 if prec == "fp64" else 1e-6) * dto
    rng = np.random.default_rng(11)
    r = 10
    # error scale: every flux term is bounded by the energy density, so each
    # cell quantity is compared against mean |e| (B against mean |B|)
    scaleU = [np.abs(U0d[4]).mean()] * 5
    scaleB = [np.abs(B0d).mean()] * 3
    for _ in range(24):
        k, j, i = rng.integers(0, 256, 3)
        u, b = neighbourhood(U0d, B0d, k, j, i, r)
        orc.step(u, b, st.dx, st.gamma, dt, integ, recon, solver)
        for f in range(5):
            assert abs(Ug[f, k, j, i] - u[f, r, r, r]) <= tol * scaleU[f], (f, k, j, i)
        for d in range(3):
            assert abs(Bg[d, k, j, i] - b[d, r, r, r]) <= tol * scaleB[d], (d, k, j, i)


@pytest.mark.parametrize("integ,recon,solver", COMBOS)
def test_invariants_on_gpu(M, integ, recon, solver):
    st = I.abc(48, kmult=2, beta=0.5, seed=7, noise=1e-2)
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, integ, recon, solver, "fp64", 0.3)
    try:
        s.set_state(st.U, st.B)
        s0 = s.sums()
        s.advance(5)
        s1 = s.sums()
        m, brms = s.divB()
        assert m / brms <= 1e-13
        scale = np.array([np.abs(st.U[f]).sum() for f in range(5)] + [np.abs(st.B[d]).sum() for d in range(3)])
        assert np.all(np.abs(s1 - s0) <= 1e-13 * scale + 1e-12)
    finally:
        s.free()


def test_deterministic_and_graph_replay(M):
    st = I.abc(40, kmult=2, beta=0.5, seed=8, noise=1e-2)
    outs = []
    for graph in (False, False, True):
        s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "ppm", "hlld", "fp64", 0.3)
        s.set_state(st.U, st.B)
        s.advance(4, use_graph=graph)
        outs.append(s.get_state())
        s.free()
    for U, B in outs[1:]:
        assert np.array_equal(U, outs[0][0]) and np.array_equal(B, outs[0][1])


def test_device_state_roundtrip_and_torch(M):
    import torch
    st = I.abc(24, kmult=1, beta=1.0, seed=9)
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", "fp64", 0.3)
    try:
        Ud = torch.from_numpy(st.U).cuda()
        Bd = torch.from_numpy(st.B).cuda()
        s.set_state(Ud, Bd)
        U2 = torch.empty_like(Ud); B2 = torch.empty_like(Bd)
        s.get_state(U2, B2)
        assert torch.equal(U2, Ud) and torch.equal(B2, Bd)
    finally:
        s.free()


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_reduced_precision_error_statement(M, prec):
    """FP32 and mixed against the FP64 oracle after 10 steps of the 32^3 ABC
    problem (same dt each step).  Stated bound on the relative L1 per field:
    1e-6 for rho, e and the face B; 3e-4 for the momentum components, whose
    values are the 1e-3 c_s velocity noise (a small denominator)."""
    tol = np.array([1e-6, 3e-4, 3e-4, 3e-4, 1e-6, 1e-6, 1e-6, 1e-6])
    st = I.abc(32, kmult=1, beta=1.0, seed=0)
    U, B = st.U.copy(), st.B.copy()
    s = M.Solver(U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", prec, 0.3)
    try:
        cast = np.float32 if prec == "fp32" else np.float64
        s.set_state(U.astype(cast), B.astype(cast))
        for _ in range(10):
            dt = orc.cfl_dt(U, B, st.dx, st.gamma, 0.3)
            s.step(dt)
            orc.step(U, B, st.dx, st.gamma, dt, "vl", "plm", "roe")
        Ug, Bg = s.get_state()
        errs = [rel_l1(Ug[f].astype(np.float64), U[f]) for f in range(5)] + \
               [rel_l1(Bg[d].astype(np.float64), B[d]) for d in range(3)]
        print(prec, ["%.2e" % e for e in errs])
        assert np.all(np.array(errs) <= tol), errs
        m, brms = s.divB()
        assert m / brms <= (1e-5 if prec == "fp32" else 1e-13)
    finally:
        s.free()


def test_negative_state_reported(M):
    st = I.abc(16, kmult=1, beta=1.0, seed=1)
    U = st.U.copy()
    U[0, 3, 4, 5] = -1.0       # planted on the host: a negative density
    s = M.Solver(U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", "fp64", 0.3)
    try:
        s.set_state(U, st.B)
        s.advance(1)
        with pytest.raises(M.MHDError) as ei:
            s.sync()
        assert ei.value.status == M.MHD_ENEGATIVE
        assert s.bad_cell() == (3 * 16 + 4) * 16 + 5
        s.clear_error()
        s.set_state(st.U, st.B)
        s.advance(1)
        s.sync()
    finally:
        s.free()


def test_bad_dt_rejected(M):
    st = I.abc(8, kmult=1)
    s = M.Solver(st.U.shape[1:], st.dx, st.gamma)
    try:
        s.set_state(st.U, st.B)
        for bad in (0.0, -1.0, float("nan"), float("inf")):
            with pytest.raises(M.MHDError) as ei:
                s.step(bad)
            assert ei.value.status == M.MHD_EINVAL
    finally:
        s.free()


def test_mixed_precision_stress_small(M):
    """The low-beta current-loop problem (beta = 1e-3, v = (2, 2, 2)) at
    64 x 32 x 32, 10 steps, against the FP64 oracle with one dt sequence.
    The thermal pressure (3.3e-4) is below the magnetic energy of the loop's
    cross term with the background (~1e-3): even the FP64 oracle reaches
    P < 0 in its first step (P_min = -9e-4), so all three run with the same
    pressure floor (1e-5, ~3 % of P0), the floored cells counted on each side.
    Stated: the mixed form keeps div B at round-off, its FP64 energy closer
    to the oracle than the FP32 form's; the per-field errors are printed."""
    pf = 1e-5
    st = I.current_loop(64, 32, 32)
    U, B = st.U.copy(), st.B.copy()
    ctx = {p: M.Solver(U.shape[1:], st.dx, st.gamma, "vl", "plm", "roe", p, 0.3, pfloor=pf) for p in ("mixed", "fp32")}
    ctx["mixed"].set_state(U, B)
    ctx["fp32"].set_state(U.astype(np.float32), B.astype(np.float32))
    nfl = 0
    for _ in range(10):
        dt = orc.cfl_dt(U, B, st.dx, st.gamma, 0.3, pfloor=pf)
        for s in ctx.values():
            s.step(dt)
        nfl += orc.step_floor(U, B, st.dx, st.gamma, dt, "vl", "plm", "roe", pfloor=pf)[1]
    W = orc.prim(U, B, st.gamma)
    res = {"oracle_floored": nfl}
    for p, s in ctx.items():
        Ug, Bg = s.get_state()
        assert np.all(np.isfinite(Ug)) and np.all(np.isfinite(Bg))
        Wg = orc.prim(Ug.astype(np.float64), Bg.astype(np.float64), st.gamma)
        res[p] = dict(rho=rel_l1(Ug[0], U[0]), e=rel_l1(Ug[4], U[4]), B=max(rel_l1(Bg[d], B[d]) for d in range(3)),
                      P=rel_l1(Wg[4], W[4]), divB=s.divB()[0] / s.divB()[1], floored=s.floor_count())
        s.free()
    print(res)
    assert res["mixed"]["divB"] <= 1e-13
    assert res["mixed"]["rho"] <= 1e-3 and res["mixed"]["e"] <= 1e-3 and res["mixed"]["B"] <= 1e-3
    assert res["mixed"]["e"] < res["fp32"]["e"]


@pytest.mark.parametrize("recon", ["plm", "ppm"])
def test_fp64_parity_roe_fallback(M, recon):
    """Two strong rarefactions (rho = 1, u = -/+2, P = 0.4, Toro's test 2) with
    a uniform oblique field along x in a 64 x 4 x 4 box: the Roe fan of the
    faces at the split has a state with P <= 0, so those faces fall back to
    HLLE (the oracle counts them).  The GPU's fan check, including its cheap
    bound that skips the check on smooth faces, must take the same decisions:
    FP64 parity at the 1e-12 bar."""
    nx, ny, nz = 64, 4, 4
    dx = 1.0 / nx
    gam = 5.0 / 3.0
    x = (np.arange(nx) + 0.5) * dx
    u = np.where((x > 0.25) & (x < 0.75), 2.0, -2.0)
    rho = np.ones((nz, ny, nx))
    vx = np.broadcast_to(u, (nz, ny, nx)).copy()
    z = np.zeros((nz, ny, nx))
    B = np.stack([np.full((nz, ny, nx), 0.5), np.full((nz, ny, nx), 0.3), np.full((nz, ny, nx), 0.2)])
    U = I.conserved(rho, vx, z, z, np.full((nz, ny, nx), 0.4), B, gam)
    st = I.State(U, B, dx, gam, {})
    Uo, Bo = U.copy(), B.copy()
    dt = orc.cfl_dt(Uo, Bo, dx, gam, 0.3)
    nfb = orc.step(Uo, Bo, dx, gam, dt, "vl", recon, "roe")
    assert nfb > 0
    run_parity(M, st, "vl", recon, "roe", 3)


def _table1(name):
    import math
    path = __file__.replace("test_gpu_parity.py", "golden/table1_riemann_states.txt")
    for line in open(path):
        if line.startswith(name + " "):
            v = [float(eval(t, {"math": math})) for t in line.split()[1:]]
            return np.array(v[0:7]), np.array(v[7:14]), v[14]
    raise KeyError(name)


@pytest.mark.parametrize("name,axis,scheme", [("torrilhon", 0, ("vl", "plm", "roe")), ("rj2a", 1, ("vl", "ppm", "hlld")),
                                              ("rj2a", 2, ("vl", "plm", "roe")), ("torrilhon", 1, ("ctu", "ppm", "hlld")),
                                              ("rj2a", 0, ("ctu", "plm", "roe"))])
def test_fp64_parity_table1_tubes(M, name, axis, scheme):
    """the Table 1 Riemann problems along x (warp sweeps), y and z (pencils),
    on a 192-cell line with 2 x 2 cells across: FP64 parity per step"""
    wl, wr, bn = _table1(name)
    st = I.shock_tube(wl, wr, bn, 192, axis=axis, m=2)
    U, B = st.U.copy(), st.B.copy()
    # first advance the oracle into the developed fan, then compare step by step
    for _ in range(20):
        dt = orc.cfl_dt(U, B, st.dx, st.gamma, 0.3)
        orc.step(U, B, st.dx, st.gamma, dt, *scheme)
    run_parity(M, I.State(U, B, st.dx, st.gamma, {}), *scheme, 4)
