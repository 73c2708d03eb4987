"""Training and evaluation of the learned path selector.

A training pair is one 4^3 block of a state: its 48 features (computed by
the library from the state) and its label, 1 when one step of the cheap
path (PLM in primitive variables + HLLE) from that state stays within tau of
one step of the full path (characteristic PPM + HLLD) on every stored field
of the block (mhd_block_error), else 0.  The states come from the method
itself: ABC fields (Eq. 20) at several wave numbers and plasma beta, ABC
fields with Sedov-type blasts, Orszag-Tang vortices (Eq. 18), the perturbed
ABC state of the relaxation run (Eqs. 21-23) and the magnetised blast with
its density noise (Eq. 19), each advanced by the full path and sampled at
several times.  The network is
trained on the GPU by the library's own forward, backward and Adam kernels.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs as I
from . import mhd

TAU = 1e-3
# pressure floor of the blast states (ambient P >= 1/30 in every training
# state); the floored cell-steps are counted and reported
PFLOOR = 1e-4
FULL = ("vl", "ppm", "hlld")
CHEAP = ("vl", "plm_prim", "hlle")


def training_ics(n=128, seed=7):
    """initial states of the training set (all n^3, FP32 stepping)"""
    rng = np.random.default_rng(seed)
    ics = []
    for kmult, beta in [(1, 1.0), (2, 0.5), (3, 0.1), (2, 0.1), (3, 1.0), (1, 0.1)]:
        ics.append(I.abc(n, kmult=kmult, beta=beta, seed=int(rng.integers(1 << 30)), noise=1e-3))
    for nb, E in [(4, 1.0), (10, 1.0), (6, 0.3)]:
        ics.append(I.abc_blasts(n, kmult=int(rng.integers(1, 4)), beta=float(rng.choice([0.1, 0.5])), nblast=nb, E=E,
                                radius=0.05, seed=int(rng.integers(1 << 30))))
    ics.append(I.orszag_tang(n, nz=n))
    # the ABC relaxation run's perturbed state (Eqs. 21-23) and the magnetised
    # blast with its density noise (Eq. 19)
    ics.append(I.abc_perturbed(n, kmult=2, beta=1.0))
    ics.append(I.mhd_blast(n, r0=0.08, theta0=85.0, phi0=45.0, density_noise=True))
    return ics


def _dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def make_pairs(ics, snapshots=(0, 4, 12, 24, 40), tau=TAU, stream=None, pfloor=PFLOOR, stats=None):
    """(X, y, err) on the device: features, labels and the block errors"""
    import torch
    Xs, ys, es = [], [], []
    nfloor = 0
    for st in ics:
        shape = st.U.shape[1:]
        full = mhd.Solver(shape, st.dx, st.gamma, *FULL, "fp32", 0.3, stream=stream, pfloor=pfloor)
        cheap = mhd.Solver(shape, st.dx, st.gamma, *CHEAP, "fp32", 0.3, stream=stream, pfloor=pfloor)
        run = mhd.Solver(shape, st.dx, st.gamma, *FULL, "fp32", 0.3, stream=stream, pfloor=pfloor)
        U = _dev(torch, st.U, torch.float32)
        B = _dev(torch, st.B, torch.float32)
        run.set_state(U, B)
        done = 0
        for snap in snapshots:
            if snap > done:
                run.advance(snap - done)
                done = snap
            run.get_state(U, B)
            full.set_state(U, B)
            cheap.set_state(U, B)
            X = full.block_features()
            dt = full.cfl_dt()
            full.step(dt)
            cheap.step(dt)
            err = mhd.block_error(full, cheap)
            Xs.append(X)
            es.append(err)
            ys.append((err <= tau).to(torch.float32))
        for s in (full, cheap, run):
            nfloor += s.floor_count()
            s.free()
    if stats is not None:
        stats["floored_cell_steps"] = nfloor
    return torch.cat(Xs), torch.cat(ys), torch.cat(es)


def class_weights(y):
    """weights that give both classes the same total weight"""
    import torch
    pos = float(y.sum().item())
    neg = float(y.numel() - pos)
    wp = 0.5 * y.numel() / max(pos, 1.0)
    wn = 0.5 * y.numel() / max(neg, 1.0)
    return torch.where(y > 0.5, torch.full_like(y, wp), torch.full_like(y, wn))


def train(X, y, epochs=4, batch=8192, lr=2e-3, seed=0, stream=None, log=None):
    """class-balanced Adam on the GPU; returns the network and the loss history"""
    import torch
    net = mhd.MLP(seed=seed, stream=stream)
    wgt = class_weights(y)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    hist = []
    n = X.shape[0]
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=g)
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            xb = X[idx].contiguous()
            yb = y[idx].contiguous()
            wb = wgt[idx].contiguous()
            want = (b0 // batch) % 20 == 0
            l = net.train_step(xb, yb, wb, lr=lr * (0.5 ** ep), want_loss=want)
            if want:
                hist.append(l)
                if log:
                    log(f"epoch {ep} batch {b0 // batch} loss {l:.4f}")
    return net, hist


def confusion(net, X, y):
    """dict: accuracy, balanced accuracy (mean of the per-class recalls),
    false-safe rate (unsafe blocks predicted safe), fraction predicted safe"""
    z = net.predict(X)
    pred = z > 0
    safe = y > 0.5
    ns = max(1.0, float(safe.float().sum().item()))
    nu = max(1.0, float((~safe).float().sum().item()))
    tpr = float((pred & safe).float().sum().item()) / ns
    tnr = float((~pred & ~safe).float().sum().item()) / nu
    return {"accuracy": float((pred == safe).float().mean().item()), "balanced_accuracy": 0.5 * (tpr + tnr),
            "false_safe": 1.0 - tnr, "predicted_safe": float(pred.float().mean().item())}


def selector_run(st, nsteps, net=None, precision="fp32", stream=None, cheap=False, pfloor=PFLOOR):
    """advance a copy of st by nsteps with the full path, the selector, or
    the cheap path everywhere; returns (state, ms per step, cheap fractions)"""
    import torch
    shape = st.U.shape[1:]
    scheme = CHEAP if cheap else FULL
    s = mhd.Solver(shape, st.dx, st.gamma, *scheme, precision, 0.3, stream=stream, pfloor=pfloor)
    s.set_state(_dev(torch, st.U, torch.float32), _dev(torch, st.B, torch.float32))
    if net is not None:
        s.set_selector(net)
    s.advance(1)
    s.sync()
    U0 = torch.empty((5, *shape), dtype=torch.float32, device="cuda")
    B0 = torch.empty((3, *shape), dtype=torch.float32, device="cuda")
    s.set_state(_dev(torch, st.U, torch.float32), _dev(torch, st.B, torch.float32))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.advance(nsteps)
    s.sync()
    ms = (time.perf_counter() - t0) * 1e3 / nsteps
    fr = s.selector_stats() if net is not None else ((1.0, 1.0) if cheap else (0.0, 0.0))
    s.get_state(U0, B0)
    s.free()
    return (U0, B0), ms, fr


def rel_l1_fields(a, b):
    """relative L1 of each of the 8 stored fields of state a against b"""
    (Ua, Ba), (Ub, Bb) = a, b
    out = [float((Ua[f] - Ub[f]).abs().sum() / Ub[f].abs().sum().clamp_min(1e-30)) for f in range(5)]
    out += [float((Ba[d] - Bb[d]).abs().sum() / Bb[d].abs().sum().clamp_min(1e-30)) for d in range(3)]
    return out
