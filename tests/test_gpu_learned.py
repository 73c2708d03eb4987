"""The learned path selector on the GPU: the training kernels' gradient
against the CPU reference network (same BF16 quantisation points), the
inference, the block features and errors against numpy restatements, the
selected step against the plain schemes it chooses between, and training
with what the network gains over the method without it."""
import numpy as np
import pytest

from oracle import mlp_oracle as R
from oracle import oracle as orc
from paper_1804_03479_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_03479_b300 import mhd
    mhd.lib()
    return torch, mhd


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def random_net(seed=0):
    rng = np.random.default_rng(seed)
    p = (rng.normal(size=R.NPARAM) * 0.15).astype(np.float32)
    return p


def test_training_gradient_matches_cpu_reference(env):
    torch, mhd = env
    rng = np.random.default_rng(1)
    n = 1000                                   # not a multiple of 16: padded rows must not count
    X = rng.normal(size=(n, 48)).astype(np.float32)
    y = (rng.random(n) < 0.35).astype(np.float32)
    w = rng.uniform(0.5, 2.0, n).astype(np.float32)
    p = random_net(2)
    net = mhd.MLP(seed=0)
    net.set_weights(p)
    g, loss = net.grad(dev(torch, X), dev(torch, y), dev(torch, w))
    g = g.cpu().numpy().astype(np.float64)
    lref, gref = R.loss_and_grad(p.astype(np.float64), X, y, w, quantise=True)
    assert abs(loss - lref) <= 1e-5 * abs(lref)
    for name, a, b in [("W1", R.P_W1, R.P_B1), ("b1", R.P_B1, R.P_W2), ("W2", R.P_W2, R.P_B2),
                       ("b2", R.P_B2, R.P_W3), ("w3", R.P_W3, R.P_B3), ("b3", R.P_B3, R.NPARAM)]:
        err = np.linalg.norm(g[a:b] - gref[a:b]) / max(np.linalg.norm(gref[a:b]), 1e-30)
        assert err <= 5e-3, (name, err)
    net.free()


def test_inference_matches_cpu_reference(env):
    torch, mhd = env
    rng = np.random.default_rng(3)
    X = rng.normal(size=(777, 48)).astype(np.float32)
    p = random_net(4)
    net = mhd.MLP()
    net.set_weights(p)
    z = net.predict(dev(torch, X)).cpu().numpy()
    zref = R.forward(p.astype(np.float64), X)["z"]
    assert np.abs(z - zref).max() <= 1e-4 * (1 + np.abs(zref).max())
    net.free()


def numpy_features(W, gam):
    """the 48 block features, restated in numpy from the cell primitives"""
    nz, ny, nx = W.shape[1:]
    out = []
    for kb in range(nz // 4):
        for jb in range(ny // 4):
            for ib in range(nx // 4):
                sl = (slice(4 * kb, 4 * kb + 4), slice(4 * jb, 4 * jb + 4), slice(4 * ib, 4 * ib + 4))
                blk = W[(slice(None),) + sl].reshape(8, -1)
                mean, sq = blk.mean(1), (blk ** 2).mean(1)
                rho, P = mean[0], max(mean[4], 1e-30)
                b2 = sq[5] + sq[6] + sq[7]
                cref = np.sqrt((gam * P + b2) / rho)
                bref = np.sqrt(b2 + P)
                scale = [rho, cref, cref, cref, P, bref, bref, bref]
                dmax = np.zeros((3, 8))
                for ax, (c0, n_ax) in enumerate([(4 * ib, nx), (4 * jb, ny), (4 * kb, nz)]):
                    idx = np.arange(c0 - 1, c0 + 5) % n_ax
                    # the slab of the block extended one cell down and up along ax
                    if ax == 0:
                        sub = W[:, sl[0], sl[1], :][:, :, :, idx]
                        d = np.abs(np.diff(sub, axis=3))
                    elif ax == 1:
                        sub = W[:, sl[0], :, sl[2]][:, :, idx, :]
                        d = np.abs(np.diff(sub, axis=2))
                    else:
                        sub = W[:, :, sl[1], sl[2]][:, idx, :, :]
                        d = np.abs(np.diff(sub, axis=1))
                    dmax[ax] = d.reshape(8, -1).max(1)
                f = []
                vabs = np.sqrt(blk[1] ** 2 + blk[2] ** 2 + blk[3] ** 2).mean()
                for q in range(8):
                    m0 = mean[q] / scale[q]
                    if q == 0:
                        m0 = np.clip(np.log10(2 * P / max(b2, 1e-30)), -6, 6) / 6
                    if q == 4:
                        m0 = vabs / cref
                    std = np.sqrt(((blk[q] - mean[q]) ** 2).mean())
                    f += [m0, (blk[q].max() - blk[q].min()) / scale[q], dmax[0, q] / scale[q], dmax[1, q] / scale[q],
                          dmax[2, q] / scale[q], std / scale[q]]
                out.append(f)
    return np.array(out)


def test_block_features_match_numpy(env):
    torch, mhd = env
    st = I.abc_blasts(16, kmult=2, beta=0.3, nblast=2, radius=0.15, seed=5, noise=1e-2)
    s = mhd.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "ppm", "hlld", "fp32", 0.3)
    s.set_state(st.U.astype(np.float32), st.B.astype(np.float32))
    f = s.block_features().cpu().numpy()
    s.free()
    W = orc.prim(st.U.astype(np.float32).astype(np.float64), st.B.astype(np.float32).astype(np.float64), st.gamma)
    ref = numpy_features(W, st.gamma)
    assert f.shape == ref.shape == (64, 48)
    assert np.allclose(f, ref, rtol=2e-4, atol=2e-5), np.abs(f - ref).max()


@pytest.mark.parametrize("shape", [(132, 8, 8), (4, 8, 12), (40, 12, 4)])
def test_block_features_match_numpy_rows(env, shape):
    """rows of 33 blocks (a warp of 32 blocks and one with a single block
    whose two x neighbours are both beyond the warp), a box one block wide
    (both neighbours wrap onto the block itself), ragged block rows"""
    torch, mhd = env
    nx, ny, nz = shape
    st = I.abc(None, kmult=1, beta=0.4, seed=9, noise=3e-2, shape=shape)
    s = mhd.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "ppm", "hlld", "fp32", 0.3)
    s.set_state(st.U.astype(np.float32), st.B.astype(np.float32))
    f = s.block_features().cpu().numpy()
    s.free()
    W = orc.prim(st.U.astype(np.float32).astype(np.float64), st.B.astype(np.float32).astype(np.float64), st.gamma)
    ref = numpy_features(W, st.gamma)
    assert f.shape == ref.shape == (nx * ny * nz // 64, 48)
    assert np.allclose(f, ref, rtol=2e-4, atol=2e-5), np.abs(f - ref).max()


def test_block_error_matches_numpy(env):
    torch, mhd = env
    st = I.abc(16, kmult=2, beta=0.5, seed=6, noise=1e-2)
    a = mhd.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "ppm", "hlld", "fp32", 0.3)
    b = mhd.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "plm_prim", "hlle", "fp32", 0.3)
    U = st.U.astype(np.float32)
    Bf = st.B.astype(np.float32)
    for s in (a, b):
        s.set_state(U, Bf)
    dt = a.cfl_dt()
    a.step(dt)
    b.step(dt)
    err = mhd.block_error(a, b).cpu().numpy()
    Ua, Ba = [x.astype(np.float64) for x in a.get_state()]
    Ub, Bb = [x.astype(np.float64) for x in b.get_state()]
    a.free(); b.free()
    g = st.gamma
    ref = []
    for kb in range(4):
        for jb in range(4):
            for ib in range(4):
                sl = (slice(4 * kb, 4 * kb + 4), slice(4 * jb, 4 * jb + 4), slice(4 * ib, 4 * ib + 4))
                qa = [Ua[f][sl] for f in range(5)] + [Ba[d][sl] for d in range(3)]
                qb = [Ub[f][sl] for f in range(5)] + [Bb[d][sl] for d in range(3)]
                bx = 0.5 * (Ba[0] + np.roll(Ba[0], -1, 2))[sl]
                by = 0.5 * (Ba[1] + np.roll(Ba[1], -1, 1))[sl]
                bz = 0.5 * (Ba[2] + np.roll(Ba[2], -1, 0))[sl]
                bsq = bx ** 2 + by ** 2 + bz ** 2
                P = ((g - 1) * (qa[4] - 0.5 * (qa[1] ** 2 + qa[2] ** 2 + qa[3] ** 2) / qa[0] - 0.5 * bsq)).mean()
                rho, e, b2 = qa[0].mean(), abs(qa[4].mean()), bsq.mean()
                cref = np.sqrt((g * P + b2) / rho)
                bref = np.sqrt(b2 + P)
                scale = [rho, rho * cref, rho * cref, rho * cref, e, bref, bref, bref]
                ref.append(max(np.abs(qa[f] - qb[f]).mean() / scale[f] for f in range(8)))
    ref = np.array(ref)
    assert np.allclose(err, ref, rtol=1e-3, atol=1e-9)
    assert ref.max() > 0


def constant_net(mhd, logit):
    p = np.zeros(R.NPARAM, np.float32)
    p[R.P_B3] = logit
    net = mhd.MLP()
    net.set_weights(p)
    return net


@pytest.mark.parametrize("mask", [0, 6, 7, 103])
@pytest.mark.parametrize("logit,scheme", [(-50.0, ("vl", "ppm", "hlld")), (50.0, ("vl", "plm_prim", "hlle"))])
def test_selector_limits_equal_plain_schemes(env, logit, scheme, mask):
    """a network that always says 'full' (or always 'cheap') must reproduce the
    plain full (or cheap) scheme bit for bit, with tile sweeps (mask 0) or
    pencil segments (the selector's segment lists) on the masked axes; with
    x by aligned marching warps (mask 103) the cheap march solves every x
    face and the full x-warp items overwrite theirs, so the always-full limit
    is the plain full scheme with its x predictor by x-warps (mask 71: the
    PPM corrector keeps its x-warps either way)"""
    torch, mhd = env
    st = I.abc_blasts(32, kmult=2, beta=0.3, nblast=2, radius=0.1, seed=8, noise=1e-2)
    U = st.U.astype(np.float32); Bf = st.B.astype(np.float32)
    plain = mhd.Solver(U.shape[1:], st.dx, st.gamma, *scheme, "fp32", 0.3)
    plain.set_sweep_pencils(71 if (mask == 103 and logit < 0) else mask, 8)
    plain.set_state(U, Bf)
    plain.advance(3)
    ref = plain.get_state()
    plain.free()
    net = constant_net(mhd, logit)
    s = mhd.Solver(U.shape[1:], st.dx, st.gamma, "vl", "ppm", "hlld", "fp32", 0.3)
    s.set_state(U, Bf)
    s.set_selector(net)
    s.set_sweep_pencils(mask, 8)     # after the selector: its lists grow with the segment count
    s.advance(3)
    got = s.get_state()
    fb, ft = s.selector_stats()
    s.free(); net.free()
    assert (fb, ft) == ((0.0, 0.0) if logit < 0 else (1.0, 1.0))
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_mixed_selection_keeps_invariants(env):
    """a random network mixes cheap and full tiles: every face flux is still
    single-valued, so conservation and div B hold"""
    torch, mhd = env
    st = I.abc_blasts(32, kmult=2, beta=0.3, nblast=3, radius=0.1, seed=9, noise=1e-2)
    net = mhd.MLP(seed=11)
    p = random_net(12)
    net.set_weights(p)
    s = mhd.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "ppm", "hlld", "fp32", 0.3)
    s.set_state(st.U.astype(np.float32), st.B.astype(np.float32))
    s0 = s.sums()
    s.set_selector(net)
    s.advance(4)
    fb, ft = s.selector_stats()
    s1 = s.sums()
    m, brms = s.divB()
    s.free(); net.free()
    assert 0.0 < ft < 1.0, (fb, ft)
    scale = np.array([np.abs(st.U[f]).sum() for f in range(5)] + [np.abs(st.B[d]).sum() for d in range(3)])
    assert np.all(np.abs(s1 - s0) <= 1e-5 * scale + 1e-6)
    assert m / brms < 1e-5


def test_training_and_gain(env):
    """train on pairs the method generates (ABC, blast, Orszag-Tang states at
    64^3), then on a held-out blast + ABC state: the network beats chance
    (balanced accuracy; training weights both classes equally, so the
    threshold favours 'full'), and the selected run is much closer to the
    all-full run than the all-cheap run while it runs a share of the tiles
    on the cheap path."""
    torch, mhd = env
    from paper_1804_03479_b300 import learned as LRN
    ics = LRN.training_ics(64, seed=3)
    X, y, err = LRN.make_pairs(ics, snapshots=(0, 4, 10, 20, 32))
    assert 0.05 < float(y.mean()) < 0.95, float(y.mean())
    net, hist = LRN.train(X, y, epochs=6, batch=4096, lr=3e-3)
    assert hist[-1] < hist[0]
    held = [I.abc_blasts(64, kmult=3, beta=0.1, nblast=6, E=1.0, radius=0.08, seed=99)]
    Xh, yh, _ = LRN.make_pairs(held, snapshots=(0, 8))
    conf = LRN.confusion(net, Xh, yh)
    print("held-out", conf, "safe fraction", float(yh.mean()))
    assert conf["balanced_accuracy"] > 0.6
    full, _, _ = LRN.selector_run(held[0], 10)
    sel, _, (fb, ft) = LRN.selector_run(held[0], 10, net=net)
    cheap, _, _ = LRN.selector_run(held[0], 10, cheap=True)
    e_sel = max(LRN.rel_l1_fields(sel, full))
    e_cheap = max(LRN.rel_l1_fields(cheap, full))
    print("cheap tile fraction", ft, "block fraction", fb, "L1 selected", e_sel, "L1 all-cheap", e_cheap)
    assert e_sel < 0.5 * e_cheap
    # a sweep tile is 32 cells long in x, so at 64^3 it runs cheap only when
    # all eight 4^3 blocks along it are predicted safe: the tile fraction is
    # far below the block fraction here (at 384^3 the two are close)
    assert fb > 0.3
    assert ft > 0.02
    net.free()


@pytest.mark.parametrize("mask", [231, 743])
@pytest.mark.parametrize("logit,scheme", [(-50.0, ("vl", "ppm", "hlld")), (50.0, ("vl", "plm_prim", "hlle"))])
def test_selector_limits_with_the_half_update_in_the_y_corrector(env, logit, scheme, mask):
    """pencil-mask 231 (bit 7): the selector's step forms the half-step state
    inside its cheap y corrector pencils, which solve every y face, the full
    list pass overwriting its faces.  743 (bit 9 as well): the cheap z
    corrector pencils also do the conservative update, after the full z list
    pass, whose faces they read.  Always 'cheap' is then the plain cheap
    scheme with the same mask bit for bit (the same kernels); always 'full'
    is the plain full scheme with the same mask to rounding (its half-step
    states come from another instantiation of the same arithmetic, its y
    faces from the PPM pencil instead of the PPM walk with the half update,
    its conservative update from the z pencils instead of the update kernel)"""
    torch, mhd = env
    st = I.abc_blasts(32, kmult=2, beta=0.3, nblast=2, radius=0.1, seed=8, noise=1e-2)
    U = st.U.astype(np.float32); Bf = st.B.astype(np.float32)
    plain = mhd.Solver(U.shape[1:], st.dx, st.gamma, *scheme, "fp32", 0.3)
    plain.set_sweep_pencils(mask if logit > 0 else mask - 32, 8)   # full: its x predictor by x-warps, as above
    plain.set_state(U, Bf)
    plain.advance(3)
    ref = plain.get_state()
    plain.free()
    net = constant_net(mhd, logit)
    s = mhd.Solver(U.shape[1:], st.dx, st.gamma, "vl", "ppm", "hlld", "fp32", 0.3)
    s.set_state(U, Bf)
    s.set_selector(net)
    s.set_sweep_pencils(mask, 8)
    assert s.launches_per_step() == 12 + 3 + 3 + 6 - 1
    s.advance(3)
    got = s.get_state()
    s.free(); net.free()
    if logit > 0:
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    else:
        for a, b in ((got[0], ref[0]), (got[1], ref[1])):
            for f in range(a.shape[0]):
                den = max(np.abs(b[f]).sum(), 1e-2 * np.abs(ref[0][0]).sum())
                assert np.abs(a[f].astype(np.float64) - b[f]).sum() / den <= 1e-5, f


def test_selector_beside_the_cheap_sweeps_graph_and_direct(env):
    """with the x predictor marching and y, z by pencils (masks 103, 231) the
    selector's passes run on their own stream beside the cheap predictor
    sweeps, which solve every face, and the full passes wait for the lists:
    a captured graph replays the same steps bit for bit as direct launches,
    with a network that mixes cheap and full blocks"""
    torch, mhd = env
    st = I.abc_blasts(32, kmult=2, beta=0.3, nblast=3, radius=0.1, seed=9, noise=1e-2)
    U = st.U.astype(np.float32); Bf = st.B.astype(np.float32)
    for mask in (103, 231, 743):
        out = []
        for graph in (False, True):
            net = mhd.MLP(seed=11)
            net.set_weights(random_net(12))
            s = mhd.Solver(U.shape[1:], st.dx, st.gamma, "vl", "ppm", "hlld", "fp32", 0.3)
            s.set_state(U, Bf)
            s.set_selector(net)
            s.set_sweep_pencils(mask, 8)
            s.advance(4, use_graph=graph)
            fb, ft = s.selector_stats()
            out.append(s.get_state())
            s.free(); net.free()
            assert 0.0 < fb < 1.0, fb
        assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1]), mask
