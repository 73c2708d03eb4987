#!/usr/bin/env python
"""Benchmark of the MHD patch advance: cell-updates/s on the 256^3 ABC box.

One step = the whole hot path: primitives + CFL dt (on the device), the
VL (or CTU) predictor sweeps, edge E, half update, corrector sweeps, edge E
and the full CT + conservative update.  Inputs are synthetic (seeded ABC
field, k = 4 pi, beta = 0.5, velocity noise 1e-3 c_s) and resident in HBM
when the timed region starts; the state (8 x 256^3 values, 537 MB in FP32)
is larger than the 126 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank advances its own replica of the box
(the path has no exchange step on one box per GPU: replicas only); the
value is the aggregate over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s at 256³ ABC MHD (FP64 plain vs FP32/learned) + HBM roofline %"
UNIT = "cell-updates/s"
PAPER_P100 = {"fp32": 1.2e8, "fp64": 5.5e7}   # Sec. 5.2 (i), Tesla P100, VL + PLM + Roe
# the step's kernel groups as the library's profiler reports them (one per
# sweep axis) and their aggregation into the seven stages of the step
AXES = ("x", "y", "z")
STAGES = ["prim_cfl", "predictor_sweeps", "emf1", "half_update", "corrector_sweeps", "emf2", "full_update"]


def stages_of(groups):
    """per-axis sweep groups summed into the seven stages"""
    out = {}
    for k, v in groups.items():
        for st in ("predictor", "corrector"):
            if k.startswith(st + "_"):
                k = st + "_sweeps"
        out[k] = out.get(k, 0.0) + v
    return {k: out[k] for k in STAGES if k in out}
SIZES = {"fp64": (8, 8, 8), "fp32": (4, 4, 4), "mixed": (4, 8, 4)}   # (rho/M, e/B, arithmetic) bytes
# Floating-point operations per face of one VL + PLM + Roe sweep launch:
# corrector = one cell's characteristic PLM reconstruction and one Roe solve,
# predictor = one Roe solve.  They are the FADD + FMUL + 2 FFMA counts that
# ncu reports for the FP32 pencil kernels at 160^3 (y sweeps: one
# reconstruction per face plus the segment's 1/32 lead-in; the Roe fan check
# skipped where its bound proves it passes), where every divide and square
# root is a single MUFU op.  The same arithmetic runs in the FP64 build, whose
# divides and square roots expand into FMA iterations (1125 executed FP64
# flops per corrector face at 128^3), so these figures serve all precisions.
# CTU: tracing = one reconstruction with characteristic tracing, the dB_n/dn
# source terms and one Roe solve per face (the y tracing pencil, 894.6);
# ctucorr = the transverse corrections of a cell's two traced states and one
# Roe solve (the y correction pencil, 523.5); FP32 at 160^3 the same way.
FLOPS_PER_FACE = {"corrector": {"fp32": 657.0, "fp64": 657.0, "mixed": 657.0},
                  "predictor": {"fp32": 393.0, "fp64": 393.0, "mixed": 393.0},
                  "tracing": {"fp32": 895.0, "fp64": 895.0, "mixed": 895.0},
                  "ctucorr": {"fp32": 524.0, "fp64": 524.0, "mixed": 524.0}}
# DRAM bytes (read + write) per face of one sweep launch, per kernel, from
# dram__bytes_read.sum + dram__bytes_write.sum of the ncu captures in
# profiles/ (FP32 at 160^3: pencil corrector 233.8 MB, pencil predictor
# 208.2 MB, x-warp corrector 219.4 MB; FP64 pencil corrector 240.0 MB at
# 128^3), scaled to other sizes by faces; a kernel changed since its capture
# has none.
TRAFFIC_PER_FACE = {"corrector_pencil": {"fp32": 58.5, "fp64": 114.4}, "predictor_pencil": {"fp32": 51.1},
                    "corrector_xwarp": {"fp32": 54.7}, "tracing_pencil": {"fp32": 111.7},
                    "tracing_xwarp": {"fp32": 113.6}, "ctucorr_pencil": {"fp32": 147.0},
                    "ctucorr_xwarp": {"fp32": 146.6}}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=d["hbm_gbs"], src="measured", sm_max_mhz=d.get("sm_max_mhz", 2032.0))
    return dict(hbm_gbs=6400.0, src="fallback", sm_max_mhz=2032.0)


def alu_peak_tflops(prec, sm_mhz):
    """dense FP32 / FP64 ALU peak from the unit counts: 148 SMs x 128 FP32
    lanes x 2 flops per FMA x clock; FP64 at the part's nominal 1.25 TFLOP/s
    scaled by the clock."""
    if prec == "fp64":
        return 1.25 * sm_mhz / 2032.0
    return 148 * 128 * 2 * sm_mhz * 1e6 / 1e12


class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1])); mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(n):
    from paper_1804_03479_b300 import inputs as I
    return I.abc(n, kmult=2, beta=0.5, seed=0)


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(torch, value, dist, device):
    """the slowest rank's time (every rank gets it); value itself when alone"""
    if not dist:
        return value
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(world, cells, steps, ms_max):
    """whole-job cell-updates/s: the units of all ranks over the slowest time"""
    return world * cells * steps / (ms_max * 1e-3)


def time_variant(torch, mhd, st, prec, scheme, K, W, dist, stream, profile=True, tune=True):
    """Device-timed steps of one precision; returns ms/step, group ms and the
    solver.  With tune, the library's autotuner first picks the sweep tiling
    (and, for VL, pencils) on this state; its choice is in s.tuned."""
    integ, recon, riemann = scheme
    cast = torch.float32 if prec == "fp32" else torch.float64
    U = torch.from_numpy(st.U).to(device="cuda", dtype=cast).contiguous()
    B = torch.from_numpy(st.B).to(device="cuda", dtype=cast).contiguous()
    s = mhd.Solver(st.U.shape[1:], st.dx, st.gamma, integ, recon, riemann, prec, 0.3, stream=stream.cuda_stream)
    s.set_state(U, B)
    del U, B
    if tune:
        s.autotune(reps=2)
    # the sweep configuration the steps run with (autotuned or the default)
    tl, bps = s.sweep_config()
    mask, plen = s.sweep_pencils()
    s.tuned = {"tile_len": tl, "blocks_per_sm": bps, "pencil_mask": mask, "pencil_len": plen,
               "autotuned": bool(tune)}
    s.advance(W)
    s.sync()
    if profile:
        s.profile_begin(K)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.advance(K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    groups, rec = s.profile_end() if profile else ({}, 0)
    s.sync()
    ms = max_over_ranks(torch, ms, dist, "cuda")
    return ms, groups, rec, s


def sweep_bytes_per_face(prec, kind="vl"):
    """algorithmic bytes per face of one sweep launch: VL (either stage) W and
    B_n in, 7 flux components out; CTU tracing the same in, the flux and the
    two traced states out; CTU correction both traced states, the cell's B_n,
    the 14 transverse fluxes and the half-step face B_n in, 7 fluxes out"""
    szu, sze, szr = SIZES[prec]
    return {"vl": 8 * szr + sze + 7 * szr, "tracing": 8 * szr + sze + 21 * szr,
            "ctucorr": 29 * szr + sze + 7 * szr}[kind]


def group_bytes(prec, n, integ="vl"):
    """algorithmic HBM bytes of each stage of one step on n cells: every
    array element a kernel needs is read once and every result written once
    (neighbour re-reads assumed to hit in cache)"""
    szu, sze, szr = SIZES[prec]
    u = 4 * szu + 4 * sze          # rho, M (TU) and e, B faces (TE)
    emf = (9 + 6 + 3) * szr        # F_rho and the two E fluxes of 3 axes, v and B_cc, E out
    s1, s2 = ("vl", "vl") if integ == "vl" else ("tracing", "ctucorr")
    return {"prim_cfl": n * (u + 8 * szr), "predictor_sweeps": 3 * n * sweep_bytes_per_face(prec, s1),
            "emf1": n * emf, "half_update": n * (u + 18 * szr + 3 * sze + 8 * szr),
            "corrector_sweeps": 3 * n * sweep_bytes_per_face(prec, s2), "emf2": n * emf,
            "full_update": n * (2 * u + 18 * szr)}


# state bytes per cell update when the state is read once and written once
# (rho, M in the arithmetic type of the form; e and the face B in FP64 for MIXED)
STATE_BYTES = {"fp64": 128, "fp32": 64, "mixed": 96}


def step_hbm(prec, n, ms_per_step, pk, integ="vl"):
    """the whole step against the HBM roofline, two ways: (1) the state read
    once and written once (the ceiling of a fully fused step), (2) the
    algorithmic bytes of this multi-kernel step (sum over the kernel groups)"""
    bpc = sum(group_bytes(prec, n, integ).values()) / n
    gbs = bpc * n / (ms_per_step * 1e-3) / 1e9
    cups = n / (ms_per_step * 1e-3)
    ceil = pk["hbm_gbs"] * 1e9 / STATE_BYTES[prec]
    return {"state_bytes_per_cell_update": STATE_BYTES[prec], "state_roofline_cell_updates_per_s": ceil,
            "frac_of_state_roofline": cups / ceil,
            "step_bytes_per_cell_update": bpc, "step_achieved_gbs": gbs, "peak_gbs": pk["hbm_gbs"],
            "frac": gbs / pk["hbm_gbs"], "peak_src": pk["src"]}


def scheme_matrix(torch, mhd, st, steps, stream, pk):
    """{CTU, VL} x {PLM, PPM} x {HLLD, Roe} x {FP64, FP32} on the same box"""
    n = int(np.prod(st.U.shape[1:]))
    out = {}
    for prec in ("fp32", "fp64"):
        k = steps if prec == "fp32" else max(2, steps // 4)
        for integ in ("ctu", "vl"):
            for recon in ("plm", "ppm"):
                for riem in ("hlld", "roe"):
                    ms, _, _, s = time_variant(torch, mhd, st, prec, (integ, recon, riem), k, 2, None, stream,
                                               profile=False, tune=prec == "fp32")
                    s.free()
                    v = n * k / (ms * 1e-3)
                    out[f"{integ}+{recon}+{riem}/{prec}"] = {
                        "value": v, "ms_per_step": ms / k, "steps": k, "sweep": s.tuned,
                        "frac_of_state_roofline": v * STATE_BYTES[prec] / (pk["hbm_gbs"] * 1e9)}
    return out


def kernels_of(groups, tuned, integ="vl"):
    """the step's launches grouped by kernel: each sweep axis belongs to the
    tile, pencil or warp kernel of its stage (from the sweep configuration;
    CTU's stages are the tracing sweeps and the corrections, per cell where
    the axis has no register form); returns {kernel: (ms summed over its
    launches, launches per step)}"""
    mask = (tuned or {}).get("pencil_mask", 0) or 0
    out = {}
    for k, v in groups.items():
        name, nl = k, 1
        for st in ("predictor", "corrector"):
            if k.startswith(st + "_"):
                d = AXES.index(k.split("_")[1])
                stage = st if integ == "vl" else ("tracing" if st == "predictor" else "ctucorr")
                other = "cell" if stage == "ctucorr" else "tile"
                name = f"{stage}_{('xwarp' if d == 0 else 'pencil') if mask >> d & 1 else other}"
        ms, cnt = out.get(name, (0.0, 0))
        out[name] = (ms + v, cnt + nl)
    return out


def roofline(prec, groups, steps, n, pk, sm_mhz, tuned=None, integ="vl"):
    """dominant kernel of the step and its achieved fraction of the roofline
    that bounds it"""
    ks = kernels_of(groups, tuned, integ)
    dom = max(ks, key=lambda k: ks[k][0])
    tot, launches = ks[dom]
    ms = tot / steps
    out = {"kernel": dom, "ms_per_step": ms, "share": tot / sum(groups.values()), "launches": launches,
           "ms_per_launch": ms / launches}
    sweep = dom.split("_")[0]
    fpf = FLOPS_PER_FACE.get(sweep, {}).get(prec)
    if sweep in ("predictor", "corrector", "tracing", "ctucorr") and fpf:
        ach = n * fpf / (ms / launches * 1e-3) / 1e12          # per launch: n faces
        peak = alu_peak_tflops(prec, sm_mhz)
        tpf = TRAFFIC_PER_FACE.get(dom, {}).get(prec)
        bpf = sweep_bytes_per_face(prec, {"tracing": "tracing", "ctucorr": "ctucorr"}.get(sweep, "vl"))
        hbm = n * bpf / (ms / launches * 1e-3) / 1e9
        out.update(bound="alu", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                   peak_src=f"{'FP64' if prec == 'fp64' else 'FP32'} peak derived from unit counts at {sm_mhz:.0f} MHz",
                   traffic=(tpf * n if tpf else None),
                   algorithmic=f"{fpf:.0f} flops per face x {n} faces per launch",
                   hbm_view={"algorithmic_bytes_per_launch": n * bpf, "achieved_gbs": hbm,
                             "frac_of_measured": hbm / pk["hbm_gbs"]})
    else:
        stage = {"emf1": "emf1", "emf2": "emf2"}.get(dom, dom)
        b = group_bytes(prec, n, integ)[stage] / launches
        ach = b / (ms / launches * 1e-3) / 1e9
        out.update(bound="hbm", achieved=ach, peak=pk["hbm_gbs"], unit="GB/s", frac=ach / pk["hbm_gbs"],
                   peak_src=pk["src"], traffic=None, algorithmic_bytes_per_launch=b)
    return out


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(scheme, target_s=12.0):
    """the FP64 oracle as it stands, all host cores, on a 64^3 sample"""
    from oracle import oracle as O
    integ, recon, riemann = scheme
    st = workload(64)
    U, B = st.U.copy(), st.B.copy()
    t0 = time.perf_counter()
    dt = O.cfl_dt(U, B, st.dx, st.gamma, 0.3)
    O.step(U, B, st.dx, st.gamma, dt, integ, recon, riemann)
    t1 = time.perf_counter() - t0
    m = max(1, min(40, int(target_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    for _ in range(m):
        dt = O.cfl_dt(U, B, st.dx, st.gamma, 0.3)
        O.step(U, B, st.dx, st.gamma, dt, integ, recon, riemann)
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": 64 ** 3 * m / el, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"64^3 ABC (k=4pi, beta=0.5, seed 0), {m} steps of {integ}+{recon}+{riemann} FP64 "
                      f"incl. the CFL dt, OpenMP on all host threads"}


def batch_variant(torch, mhd, K, stream):
    """The batched uneven workload: 48 independent periodic boxes with sides
    drawn from {32, 48, 64, 96, 128, 192} (seed 1), linear waves and ABC
    fields in turn, FP32 VL + PPM + HLLD.  One graph-captured batched step
    (every kernel stage one launch over all boxes, autotuned sweep tiling)
    against a loop that steps each box on its own context."""
    from paper_1804_03479_b300 import inputs as I
    sides = I.box_sides(48, seed=1)
    boxes = [I.batch_box(i, sd, seed=1) for i, sd in enumerate(sides)]
    shapes = [b.U.shape[1:] for b in boxes]
    dxs = [b.dx for b in boxes]
    ncell = sum(int(np.prod(sh)) for sh in shapes)
    s = mhd.Solver(None, None, 5 / 3, "vl", "ppm", "hlld", "fp32", 0.3, stream=stream.cuda_stream,
                   shapes=shapes, dxs=dxs)
    for k, b in enumerate(boxes):
        s.set_state(torch.from_numpy(b.U).to("cuda", torch.float32), torch.from_numpy(b.B).to("cuda", torch.float32), box=k)
    tl, bps, tune_ms = s.autotune(reps=2)
    s.advance(2, use_graph=True)
    s.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.advance(K, use_graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    s.sync()
    s.free()
    # the same boxes, one context each, stepped one after the other
    ctxs = []
    for b in boxes:
        c = mhd.Solver(b.U.shape[1:], b.dx, 5 / 3, "vl", "ppm", "hlld", "fp32", 0.3, stream=stream.cuda_stream)
        c.set_state(torch.from_numpy(b.U).to("cuda", torch.float32), torch.from_numpy(b.B).to("cuda", torch.float32))
        ctxs.append(c)
    for c in ctxs:
        c.advance(1)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(K):
        for c in ctxs:
            c.advance(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_loop = e0.elapsed_time(e1) / K
    for c in ctxs:
        c.free()
    return {"value": ncell / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": K, "boxes": 48,
            "cells": ncell, "sides": sides, "scheme": "vl+ppm+hlld", "precision": "fp32",
            "sweep_tiling": {"tile_len": tl, "blocks_per_sm": bps, "autotune_ms_per_step": tune_ms},
            "launches_per_step": 12, "graph": True,
            "per_box_loop": {"value": ncell / (ms_loop * 1e-3), "ms_per_step": ms_loop, "launches_per_step": 12 * 48},
            "speedup_vs_per_box_loop": ms_loop / ms}


def learned_variant(torch, mhd, K, stream):
    """The learned path select on the 384^3 ABC box (k = 6 pi, beta = 0.1) with
    ten seeded Sedov-type blasts (E = 1 in r < 0.05): the selector network is
    trained here on pairs the method generates at 128^3 (ABC, blast and
    Orszag-Tang states), then the selected FP32 VL run is timed against the
    all-full (PPM + HLLD) run from the same state, with the L1 difference
    after K steps per field."""
    from paper_1804_03479_b300 import inputs as I
    from paper_1804_03479_b300 import learned as LRN
    t0 = time.perf_counter()
    stats = {}
    X, y, err = LRN.make_pairs(LRN.training_ics(128, seed=7), stats=stats)
    net, hist = LRN.train(X, y, epochs=4, batch=8192, lr=2e-3)
    conf_train = LRN.confusion(net, X, y)
    t_train = time.perf_counter() - t0
    npairs, safe = int(X.shape[0]), float(y.mean().item())
    del X, y, err
    st = I.abc_blasts(384, kmult=3, beta=0.1, nblast=10, E=1.0, radius=0.05, seed=2)
    Xh, yh, _ = LRN.make_pairs([st], snapshots=(0,))
    conf_held = LRN.confusion(net, Xh, yh)
    del Xh, yh
    out = {}
    states = {}
    for name in ("full", "selected"):
        s = mhd.Solver(st.U.shape[1:], st.dx, st.gamma, *LRN.FULL, "fp32", 0.3, stream=stream.cuda_stream,
                       pfloor=LRN.PFLOOR)
        U = torch.from_numpy(st.U).to("cuda", torch.float32)
        B = torch.from_numpy(st.B).to("cuda", torch.float32)
        if name == "selected":
            s.set_selector(net)
        s.set_state(U, B)
        s.advance(2)                      # warm-up, then back to the initial state
        s.set_state(U, B)
        s.sync()
        s.profile_begin(K)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.advance(K)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / K
        groups, rec = s.profile_end()
        if name == "selected":
            out["cheap_fraction_blocks"], out["cheap_fraction_tiles"] = s.selector_stats()
        s.get_state(U, B)
        states[name] = (U, B)
        out[name] = {"value": st.U[0].size / (ms * 1e-3), "ms_per_step": ms,
                     "kernel_ms_per_step": {k: v / rec for k, v in stages_of(groups).items()},
                     "floored_cell_steps": s.floor_count()}
        s.free()
    net.free()
    l1 = LRN.rel_l1_fields(states["selected"], states["full"])
    return {"value": out["selected"]["value"], "unit": UNIT, "ms_per_step": out["selected"]["ms_per_step"],
            "steps": K, "workload": "abc384_k6pi_beta0.1 + 10 blasts (E=1, r<0.05, seed 2)",
            "precision": "fp32", "full_path": out["full"], "selected_path": out["selected"],
            "speedup_vs_all_full": out["full"]["ms_per_step"] / out["selected"]["ms_per_step"],
            "cheap_fraction_blocks": out["cheap_fraction_blocks"], "cheap_fraction_tiles": out["cheap_fraction_tiles"],
            "rel_l1_vs_all_full_after_steps": dict(zip(["rho", "Mx", "My", "Mz", "e", "Bx", "By", "Bz"], l1)),
            "tau": LRN.TAU, "pfloor": LRN.PFLOOR,
            "training": {"pairs": npairs, "safe_fraction": safe, "wall_s": t_train, "train": conf_train,
                         "held_out_384": conf_held, "loss_first_last": [hist[0], hist[-1]],
                         "floored_cell_steps": stats.get("floored_cell_steps")}}


def e2e(torch, mhd, st, prec, scheme, K, stream, nstreams=2):
    """same metric through the C ABI with host buffers: each step copies the
    state in from pinned host memory (mhd_set_state), advances one step
    (mhd_advance) and copies the state back out (mhd_get_state).  With
    nstreams > 1, as many contexts run on their own CUDA streams from as many
    host threads (the calls release the GIL), so one context's copies
    overlap another's step; every step still carries its own copies."""
    import threading
    integ, recon, riemann = scheme
    cast = torch.float32 if prec == "fp32" else torch.float64
    Uh = torch.from_numpy(st.U).to(dtype=cast).pin_memory()
    Bh = torch.from_numpy(st.B).to(dtype=cast).pin_memory()
    n = st.U[0].size
    nbytes = Uh.numel() * Uh.element_size() + Bh.numel() * Bh.element_size()

    def run(ns, steps):
        ctxs = []
        for q in range(ns):
            sq = torch.cuda.Stream()
            s = mhd.Solver(st.U.shape[1:], st.dx, st.gamma, integ, recon, riemann, prec, 0.3,
                           stream=sq.cuda_stream)
            Uo = torch.empty_like(Uh).pin_memory()
            Bo = torch.empty_like(Bh).pin_memory()
            s.set_state(Uh, Bh)
            s.advance(1)
            s.get_state(Uo, Bo)
            ctxs.append((s, Uo, Bo, sq))
        torch.cuda.synchronize()
        each = max(1, steps // ns)

        def work(s, Uo, Bo):
            for _ in range(each):
                s.set_state(Uh, Bh)
                s.advance(1)
                s.get_state(Uo, Bo)

        th = [threading.Thread(target=work, args=c[:3]) for c in ctxs]
        t0 = time.perf_counter()
        for t in th:
            t.start()
        for t in th:
            t.join()
        el = time.perf_counter() - t0
        for c in ctxs:
            c[0].free()
        return n * each * ns / el, each * ns

    def link(reps=6):
        """the same bytes copied in both directions at once with no step
        between them: the host link's bound on this metric"""
        dU, dB = torch.empty_like(Uh, device="cuda"), torch.empty_like(Bh, device="cuda")
        sU, sB = torch.empty_like(dU), torch.empty_like(dB)
        oU, oB = torch.empty_like(Uh).pin_memory(), torch.empty_like(Bh).pin_memory()
        up, down = torch.cuda.Stream(), torch.cuda.Stream()

        def once():
            with torch.cuda.stream(up):
                dU.copy_(Uh, non_blocking=True)
                dB.copy_(Bh, non_blocking=True)
            with torch.cuda.stream(down):
                oU.copy_(sU, non_blocking=True)
                oB.copy_(sB, non_blocking=True)

        once()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            once()
        torch.cuda.synchronize()
        el = (time.perf_counter() - t0) / reps
        del dU, dB, sU, sB
        return n / el, 2 * nbytes / el / 1e9

    serial, _ = run(1, K)
    value, done = run(nstreams, K) if nstreams > 1 else (serial, K)
    bound, gbs = link()
    return {"value": value, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "steps": done, "streams": nstreams, "one_stream_value": serial,
            "copy_only_bound": bound, "link_gbs_both_directions": gbs, "frac_of_copy_bound": value / bound,
            "path": "mhd_set_state(host) + mhd_advance(1) + mhd_get_state(host), "
                    f"{nstreams} contexts on their own streams and host threads"}


def run_stress(args):
    """Mixed-precision stress: 512 x 256 x 256 (a 2 x 1 x 1 box, dx = 1/256)
    low-beta ABC field (beta = 1e-3, rho = 1) plus a current loop
    (A_z = 1e-3 (0.3 - r), r < 0.3) carried at v = (2, 2, 2).  The FP64,
    MIXED and FP32 forms (VL + PLM + Roe) advance the same initial state with
    one dt sequence (the FP64 run's CFL dt each step); reported: relative L1
    per field of MIXED and FP32 against FP64 (the FP64 path matches the CPU
    oracle to 1e-12 per step) and max |div B| dx / B_rms of each form.  The
    thermal pressure is below the loop's magnetic cross term, and the FP64
    scheme itself reaches P < 0 within a step, so every form runs with the
    same pressure floor (--stress-pfloor) and reports its floored cell-steps."""
    import torch
    from paper_1804_03479_b300 import build as Bld
    Bld.build()
    from paper_1804_03479_b300 import inputs as I
    from paper_1804_03479_b300 import mhd
    torch.cuda.set_device(0)
    nx, ny, nz = args.stress_shape
    st = I.current_loop(nx, ny, nz)
    pf = args.stress_pfloor
    forms = {}
    for prec in ("fp64", "mixed", "fp32"):
        cast = torch.float32 if prec == "fp32" else torch.float64
        s = mhd.Solver(st.U.shape[1:], st.dx, st.gamma, args.integrator, args.recon, args.riemann, prec, 0.3,
                       pfloor=pf)
        s.set_state(torch.from_numpy(st.U).to("cuda", cast), torch.from_numpy(st.B).to("cuda", cast))
        forms[prec] = s
    t0 = time.perf_counter()
    for _ in range(args.stress_steps):
        dt = forms["fp64"].cfl_dt()
        for s in forms.values():
            s.step(dt)
    for s in forms.values():
        s.sync()
    wall = time.perf_counter() - t0
    ref = forms["fp64"].get_state()
    names = ["rho", "Mx", "My", "Mz", "e", "Bx", "By", "Bz"]
    out = {}
    for prec, s in forms.items():
        U, B = s.get_state()
        m, r = s.divB()
        entry = {"max_divB_dx_over_Brms": m / r, "floored_cell_steps": s.floor_count(),
                 "finite": bool(np.all(np.isfinite(U)) and np.all(np.isfinite(B)))}
        if prec != "fp64":
            l1 = [float(np.abs(U[f].astype(np.float64) - ref[0][f]).sum() / np.abs(ref[0][f]).sum()) for f in range(5)]
            l1 += [float(np.abs(B[d].astype(np.float64) - ref[1][d]).sum() / np.abs(ref[1][d]).sum()) for d in range(3)]
            entry["rel_l1_vs_fp64"] = dict(zip(names, l1))
        out[prec] = entry
        s.free()
    line = {"mode": "precision_stress", "workload": f"current loop on low-beta ABC, {nx}x{ny}x{nz}, beta=1e-3, v=(2,2,2)",
            "scheme": f"{args.integrator}+{args.recon}+{args.riemann}", "steps": args.stress_steps, "wall_s": wall,
            "pfloor": pf, "cells": nx * ny * nz, "forms": out}
    print(json.dumps(line), flush=True)


def run_reference(args):
    ws, rank, local = dist_info()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    scheme = (args.integrator, args.recon, args.riemann)
    st = workload(64)
    U, B = st.U.copy(), st.B.copy()
    for _ in range(args.warmup):
        dt = O.cfl_dt(U, B, st.dx, st.gamma, 0.3)
        O.step(U, B, st.dx, st.gamma, dt, *scheme)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        dt = O.cfl_dt(U, B, st.dx, st.gamma, 0.3)
        O.step(U, B, st.dx, st.gamma, dt, *scheme)
    el = time.perf_counter() - t0
    v = 64 ** 3 * args.steps / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"each step one FP64 oracle step ({'+'.join(scheme)}, CFL dt included) on a 64^3 sample of the "
              f"256^3 ABC workload family (k=4pi, beta=0.5, seed 0), OpenMP on all host threads")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "abc256_k4pi_beta0.5 (64^3 sample per step)", "scheme": "+".join(scheme)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "mixed"])
    ap.add_argument("--integrator", default="vl")
    ap.add_argument("--recon", default="plm")
    ap.add_argument("--riemann", default="roe")
    ap.add_argument("--variants", default="fp64,mixed", help="other precisions measured beside the main line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-matrix", action="store_true", help="skip the 16 scheme x precision combinations")
    ap.add_argument("--no-autotune", action="store_true", help="default sweep tiling instead of the autotuned one")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--stress", action="store_true", help="mixed-precision stress run (not a bench line)")
    ap.add_argument("--stress-steps", type=int, default=500)
    ap.add_argument("--stress-shape", type=int, nargs=3, default=[512, 256, 256])
    ap.add_argument("--stress-pfloor", type=float, default=1e-5)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.stress:
        return run_stress(args)

    import torch
    from paper_1804_03479_b300 import build as Bld
    Bld.build()
    from paper_1804_03479_b300 import mhd

    ws, rank, local = dist_info()
    dist = None
    if ws > 1:
        import torch.distributed as td
        torch.cuda.set_device(local)
        td.init_process_group("nccl")
        dist = td
    else:
        torch.cuda.set_device(0)
    pk = peaks()
    scheme = (args.integrator, args.recon, args.riemann)
    st = workload(args.n)
    n = args.n ** 3
    stream = torch.cuda.Stream()
    clk = Clocks(local)
    clk.start()
    ms, groups, rec, s = time_variant(torch, mhd, st, args.precision, scheme, args.steps, args.warmup, dist, stream,
                                      tune=not args.no_autotune)
    clocks = clk.stop()
    launches = s.launches_per_step() * args.steps
    dev_bytes = s.device_bytes()
    s.free()
    sm_mhz = clocks["sm_mhz"] if clocks else pk["sm_max_mhz"]
    value = aggregate_value(ws, n, args.steps, ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_P100[args.precision] if args.precision in PAPER_P100 else None,
        "dtype": {"fp32": "f32", "fp64": "f64", "mixed": "f32+f64"}[args.precision],
        "data": "synthetic (seeded ABC field, k=4pi, beta=0.5, velocity noise 1e-3 c_s)",
        "config": {"workload": f"abc{args.n}_k4pi_beta0.5", "grid": [args.n] * 3, "scheme": "+".join(scheme),
                   "precision": args.precision, "cfl": 0.3, "dt": "CFL on device every step",
                   "l2": "state larger than L2 (no flush)", "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU",
                   "device_bytes": dev_bytes, "sweep": s.tuned},
        "roofline": roofline(args.precision, groups, rec, n, pk, sm_mhz, s.tuned, args.integrator) if rec else None,
        "hbm_roofline_step": step_hbm(args.precision, n, ms / args.steps, pk, args.integrator),
        "kernel_ms_per_step": {k: v / rec for k, v in stages_of(groups).items()} if rec else None,
        "sweep_ms_per_step": {k: v / rec for k, v in groups.items() if "_" in k and k.split("_")[1] in AXES}
        if rec else None,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rank == 0:
        variants = {}
        for prec in [p for p in args.variants.split(",") if p and p != args.precision]:
            kv = max(3, min(args.steps, 10))
            msv, gv, recv, sv = time_variant(torch, mhd, st, prec, scheme, kv, 2, None, stream,
                                             tune=not args.no_autotune)
            sv.free()
            vv = n * kv / (msv * 1e-3)
            variants[prec] = {"value": vv, "unit": UNIT, "ms_per_step": msv / kv, "steps": kv,
                              "vs_p100_paper": vv / PAPER_P100[prec] if prec in PAPER_P100 else None,
                              "roofline": roofline(prec, gv, recv, n, pk, sm_mhz, sv.tuned, args.integrator)
                              if recv else None,
                              "hbm_roofline_step": step_hbm(prec, n, msv / kv, pk, args.integrator),
                              "kernel_ms_per_step": {k: v / recv for k, v in stages_of(gv).items()} if recv else None,
                              "sweep": sv.tuned}
        if not args.no_matrix:
            variants["schemes256"] = scheme_matrix(torch, mhd, st, max(3, min(args.steps, 10)), stream, pk)
        if not args.no_batch:
            variants["batch48"] = batch_variant(torch, mhd, max(3, min(args.steps, 10)), stream)
        if not args.no_learned:
            variants["learned384"] = learned_variant(torch, mhd, max(3, min(args.steps, 10)), stream)
        line["variants"] = variants
        if not args.no_e2e:
            line["e2e"] = e2e(torch, mhd, st, args.precision, scheme, max(4, min(args.steps, 16)), stream)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(scheme)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
