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
STAGES = ["prim_cfl", "predictor_yprim", "predictor_fused", "predictor_sweeps", "emf1", "half_update", "corrector_yhalf",
          "corrector_sweeps", "corrector_zfull", "emf2", "full_update"]


def is_fused(tuned, integ="vl"):
    """the VL predictor runs as one kernel (pencil-mask bit 3; periodic boxes)"""
    return integ == "vl" and bool(((tuned or {}).get("pencil_mask", 0) or 0) & 8)


def is_yhalf(tuned, integ="vl", recon="plm"):
    """the VL half update runs inside the y corrector pencils (pencil-mask
    bits 1 and 7, bit 3 clear; periodic boxes)"""
    m = (tuned or {}).get("pencil_mask", 0) or 0
    return integ == "vl" and (m & 130) == 130 and not m & 8


def is_yprim(tuned, integ="vl", pfloor=0.0):
    """the t^n primitives and CFL speeds run inside the y predictor pencils
    (pencil-mask bits 1 and 8, bit 3 clear, no pressure floor; periodic)"""
    m = (tuned or {}).get("pencil_mask", 0) or 0
    return integ == "vl" and (m & 258) == 258 and not m & 8 and not pfloor > 0


def is_zfull(tuned, integ="vl", recon="plm"):
    """the conservative full update runs inside the z corrector pencils and
    the full-update group times the CT kernel (pencil-mask bits 2 and 9, a
    PLM reconstruction, bit 3 clear; periodic boxes)"""
    m = (tuned or {}).get("pencil_mask", 0) or 0
    return integ == "vl" and recon != "ppm" and (m & 516) == 516 and not m & 8


def fold_groups(groups, tuned, integ="vl", recon="plm", pfloor=0.0):
    """With the fused VL predictor the library's half-update group times the
    fused kernel, and the predictor-sweep and first edge-field groups are
    empty (back-to-back events): name the group for what it ran.  With the
    half update inside the y corrector pencils the half-update group times
    that kernel and the y corrector group is empty: corrector_yhalf.  With
    the primitives inside the y predictor pencils the primitive group times
    that kernel and the y predictor group is empty: predictor_yprim.  With
    the conservative full update inside the z corrector pencils the z
    corrector group is corrector_zfull (the full-update group is then CT
    alone)."""
    yp, yh = is_yprim(tuned, integ, pfloor), is_yhalf(tuned, integ, recon)
    zf = is_zfull(tuned, integ, recon)
    if yp or yh or zf:
        out = dict(groups)
        if yp:
            out["predictor_yprim"] = out.pop("prim_cfl", 0.0) + out.pop("predictor_y", 0.0)
        if yh:
            out["corrector_yhalf"] = out.pop("half_update", 0.0) + out.pop("corrector_y", 0.0)
        if zf:
            out["corrector_zfull"] = out.pop("corrector_z", 0.0)
        return out
    if not is_fused(tuned, integ):
        return groups
    out = {k: v for k, v in groups.items() if not (k.startswith("predictor_") or k == "emf1")}
    out["predictor_fused"] = out.pop("half_update", 0.0)
    return out


def stages_of(groups):
    """per-axis sweep groups summed into the seven stages"""
    out = {}
    for k, v in groups.items():
        for st in ("predictor", "corrector"):
            if k.startswith(st + "_") and k.split("_")[1] in AXES:
                k = st + "_sweeps"
        out[k] = out.get(k, 0.0) + v
    return {k: out[k] for k in STAGES if k in out}
SIZES = {"fp64": (8, 8, 8), "fp32": (4, 4, 4), "mixed": (4, 8, 4)}   # (rho/M, e/B, arithmetic) bytes
# EXECUTED floating-point operations per face of the FP32 sweep kernels: the
# FADD + FMUL + 2 FFMA counts ncu reports for the pencil kernels at 160^3
# (corrector = one characteristic PLM reconstruction and one Roe solve,
# predictor = one Roe solve; CTU tracing and correction pencils likewise),
# every divide and square root a single MUFU op.  These are what the
# kernels run, after their exact identities (one-sided Roe flux, sparse
# eigenvectors, the fan-check bound); the ALGORITHMIC counts of the method
# come from the oracle (oracle/flops_per_cell.json) and are the roofline's
# numerator.
EXEC_FLOPS_PER_FACE = {"corrector": 670.0, "predictor": 393.0, "tracing": 895.0, "ctucorr": 524.0}
# DRAM bytes (read + write) per face of one sweep launch, per kernel, from
# dram__bytes_read.sum + dram__bytes_write.sum of the ncu captures in
# profiles/ (FP32 at 160^3 for 4,096,000 faces: the y corrector with the
# half update 727.6 MB (one face and one half-step state per cell), pencil corrector 234.7 MB,
# x-march corrector 225.5 MB, x-warp corrector 225.8 MB, pencil predictor
# 208.0 MB, staged x-march predictor 204.7 MB), scaled to other sizes by
# faces.  A kernel changed since its capture has none (CTU tracing and the
# FP64 forms were re-built since theirs).
TRAFFIC_PER_FACE = {"corrector_yhalf": {"fp32": 177.6},      # per cell (727.6 MB for 4,096,000 cells)
                    "corrector_zfull": {"fp32": 127.0},      # per cell (520.2 MB)
                    "corrector_pencil": {"fp32": 57.3}, "corrector_xmarch": {"fp32": 55.0},
                    "predictor_pencil": {"fp32": 50.8}, "predictor_xmarch": {"fp32": 50.0},
                    "corrector_xwarp": {"fp32": 55.1},
                    "ctucorr_pencil": {"fp32": 147.0}, "ctucorr_xwarp": {"fp32": 146.6}}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=d["hbm_gbs"], src="measured", sm_max_mhz=d.get("sm_max_mhz", 2032.0))
    return dict(hbm_gbs=6400.0, src="fallback", sm_max_mhz=2032.0)


def alu_peaks(mhd):
    """FP32 and FP64 FMA throughput measured on this device now
    (mhd_fma_peak: best of 5 launches of independent FMA chains, CUDA events,
    at the clocks the device runs); the arithmetic roofline's peak"""
    return {"fp32": mhd.fma_peak("fp32", 5), "fp64": mhd.fma_peak("fp64", 5),
            "src": "measured by mhd_fma_peak in this run"}


def alu_peak_of(prec, apk):
    """MIXED runs its arithmetic in FP32 (FP64 only per cell: pressure, CT)"""
    return apk["fp64"] if prec == "fp64" else apk["fp32"]


FLOP_TABLE = os.path.join(ROOT, "oracle", "flops_per_cell.json")
_flop_table = None


def flop_table():
    """the oracle's operation counts per cell-update, per scheme and stage
    (written by oracle/flops.py from the oracle's own source compiled with a
    counting scalar type; read here as data)"""
    global _flop_table
    if _flop_table is None:
        with open(FLOP_TABLE) as fh:
            _flop_table = json.load(fh)
    return _flop_table


def alg_flops(scheme, kind="nontrivial"):
    """per-stage algorithmic flops per cell-update of one scheme, with the
    sweep stages also per face (three faces per cell-update)"""
    c = flop_table()["combos"]["-".join(scheme)]
    f = {k: v[kind] for k, v in c.items()}
    integ = scheme[0]
    if integ == "vl":
        per_face = {"predictor": f["riemann_predictor"] / 3,
                    "corrector": (f["reconstruction"] + f["riemann_corrector"]) / 3}
    else:
        per_face = {"tracing": (f["reconstruction_tracing"] + f["riemann_predictor"]) / 3,
                    "ctucorr": (f["transverse_correction"] + f["riemann_corrector"]) / 3}
    # per cell of the per-cell kernel groups: the primitive pass is counted
    # twice in the step (t^n with the CFL maximum, t^{n+1/2} in the half update)
    per_cell = {"prim_cfl": f["primitives"] / 2 + f["cfl"], "emf1": f["edge_emf"] / 2,
                "emf2": f["edge_emf"] / 2, "half_update": f["half_update"] + f["primitives"] / 2,
                "full_update": f["full_update"]}
    return {"total": f["total"], "per_face": per_face, "per_cell": per_cell}


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


def time_variant(torch, mhd, st, prec, scheme, K, W, dist, stream, profile=True, tune=True, forms=None):
    """Device-timed steps of one precision; returns ms/step, group ms and the
    solver.  With tune, the library's autotuner first picks the sweep tiling
    (and, for VL, pencils) on this state; its choice is in s.tuned.  forms:
    an explicit (pencil_mask, pencil_len, emf_staging), entries None for the
    autotuned or default choice."""
    integ, recon, riemann = scheme
    cast = torch.float32 if prec == "fp32" else torch.float64
    U = torch.from_numpy(st.U).to(device="cuda", dtype=cast).contiguous()
    B = torch.from_numpy(st.B).to(device="cuda", dtype=cast).contiguous()
    s = mhd.Solver(st.U.shape[1:], st.dx, st.gamma, integ, recon, riemann, prec, 0.3, stream=stream.cuda_stream)
    s.set_state(U, B)
    del U, B
    if tune:
        s.autotune(reps=2)
    if forms is not None:
        fm, fl, fe = forms
        if fm is not None or fl is not None:
            m0, l0 = s.sweep_pencils()
            s.set_sweep_pencils(m0 if fm is None else fm, l0 if fl is None else fl)
        if fe is not None:
            s.set_emf_staging(fe)
    # the sweep configuration the steps run with (autotuned or the default)
    tl, bps = s.sweep_config()
    mask, plen = s.sweep_pencils()
    s.tuned = {"tile_len": tl, "blocks_per_sm": bps, "pencil_mask": mask, "pencil_len": plen,
               "emf_staging": s.emf_staging()[1], "autotuned": bool(tune)}
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
    groups = fold_groups(groups, s.tuned, integ, recon)
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


def group_bytes(prec, n, integ="vl", fused=False, yhalf=False, yprim=False, zfull=False):
    """algorithmic HBM bytes of each stage of one step on n cells: every
    array element a kernel needs is read once and every result written once
    (neighbour re-reads assumed to hit in cache).  The fused VL predictor
    reads W, the face field and rho, M, e and writes Bh and Wh.  The y
    corrector with the half update reads what the half update reads and
    writes what it writes, plus the 7 y fluxes; the y predictor with the
    primitives reads and writes what the primitive pass does, plus the 7 y
    fluxes; the z corrector with the conservative update reads W and B_n, rho,
    M, e and the x and y fluxes' 10 hydrodynamic components and writes rho, M,
    e and 3 z flux components, and the CT update that follows reads E and B
    and writes B."""
    szu, sze, szr = SIZES[prec]
    u = 4 * szu + 4 * sze          # rho, M (TU) and e, B faces (TE)
    emf = (9 + 6 + 3) * szr        # F_rho and the two E fluxes of 3 axes, v and B_cc, E out
    s1, s2 = ("vl", "vl") if integ == "vl" else ("tracing", "ctucorr")
    out = {"prim_cfl": n * (u + 8 * szr), "predictor_sweeps": 3 * n * sweep_bytes_per_face(prec, s1),
           "emf1": n * emf, "half_update": n * (u + 18 * szr + 3 * sze + 8 * szr),
           "corrector_sweeps": 3 * n * sweep_bytes_per_face(prec, s2), "emf2": n * emf,
           "full_update": n * (2 * u + 18 * szr)}
    if fused:
        for k in ("predictor_sweeps", "emf1", "half_update"):
            del out[k]
        out["predictor_fused"] = n * (8 * szr + u + 3 * sze + 8 * szr)
    else:
        if yhalf:
            out["corrector_yhalf"] = out.pop("half_update") + n * 7 * szr
            out["corrector_sweeps"] = 2 * n * sweep_bytes_per_face(prec, s2)
        if yprim:
            out["predictor_yprim"] = out.pop("prim_cfl") + n * 7 * szr
            out["predictor_sweeps"] = 2 * n * sweep_bytes_per_face(prec, s1)
        if zfull:
            out["corrector_zfull"] = n * (8 * szr + sze + 3 * szr + 2 * (4 * szu + sze) + 10 * szr)
            out["corrector_sweeps"] -= n * sweep_bytes_per_face(prec, s2)
            out["full_update"] = n * (3 * szr + 6 * sze)
    return out


# state bytes per cell update when the state is read once and written once
# (rho, M in the arithmetic type of the form; e and the face B in FP64 for MIXED)
STATE_BYTES = {"fp64": 128, "fp32": 64, "mixed": 96}


def step_roofline(prec, n, ms_per_step, pk, apk, scheme, flops_per_cell=None, fused=False, yhalf=False,
                  yprim=False, zfull=False):
    """The whole step against its two ceilings, both from the method, not
    from this implementation's kernel split: HBM (the state read once and
    written once: 64 / 96 / 128 B per cell-update) and the arithmetic pipe
    (the oracle-counted algorithmic flops per cell-update over the measured
    FMA peak).  The lower ceiling binds; frac = value / that ceiling.  The
    multi-kernel step's own global traffic (design bytes) is reported beside
    it, not as a roofline."""
    cups = n / (ms_per_step * 1e-3)
    hbm_ceil = pk["hbm_gbs"] * 1e9 / STATE_BYTES[prec]
    fl = flops_per_cell if flops_per_cell is not None else alg_flops(scheme)["total"]
    fl_raw = alg_flops(scheme, "flops")["total"] if flops_per_cell is None else None
    alu_peak = alu_peak_of(prec, apk)
    alu_ceil = alu_peak * 1e12 / fl
    bound = "alu" if alu_ceil < hbm_ceil else "hbm"
    design = sum(group_bytes(prec, n, scheme[0], fused, yhalf, yprim, zfull).values()) / n
    return {"bound": bound, "frac": cups / min(alu_ceil, hbm_ceil),
            "hbm": {"bytes_per_cell_update": STATE_BYTES[prec], "ceiling_cell_updates_per_s": hbm_ceil,
                    "frac": cups / hbm_ceil, "peak_gbs": pk["hbm_gbs"], "peak_src": pk["src"]},
            "alu": {"flops_per_cell_update": fl, "flops_per_cell_update_with_trivial": fl_raw,
                    "ceiling_cell_updates_per_s": alu_ceil, "frac": cups / alu_ceil, "peak_tflops": alu_peak,
                    "peak_src": apk["src"], "flops_src": "oracle count, nontrivial operations"},
            "design_bytes_per_cell_update": design,
            "design_bytes_achieved_gbs": design * cups / 1e9}


def scheme_matrix(torch, mhd, st, steps_fp32, steps_fp64, stream, pk, apk):
    """{CTU, VL} x {PLM, PPM} x {HLLD, Roe} x {FP64, FP32} on the same box.
    FP32 runs the 100 steps of the 256^3 workload's statement; FP64 (15-40 x
    slower, bound by the FP64 rate) fewer, so that the default run stays
    within minutes."""
    n = int(np.prod(st.U.shape[1:]))
    out = {}
    for prec in ("fp32", "fp64"):
        k = steps_fp32 if prec == "fp32" else steps_fp64
        for integ in ("ctu", "vl"):
            for recon in ("plm", "ppm"):
                for riem in ("hlld", "roe"):
                    ms, _, _, s = time_variant(torch, mhd, st, prec, (integ, recon, riem), k, 2, None, stream,
                                               profile=False, tune=prec == "fp32")
                    s.free()
                    v = n * k / (ms * 1e-3)
                    out[f"{integ}+{recon}+{riem}/{prec}"] = {
                        "value": v, "ms_per_step": ms / k, "steps": k, "sweep": s.tuned,
                        "step_roofline": step_roofline(prec, n, ms / k, pk, apk, (integ, recon, riem),
                                                       fused=is_fused(s.tuned, integ),
                                                       yhalf=is_yhalf(s.tuned, integ, recon),
                                                       yprim=is_yprim(s.tuned, integ),
                                                       zfull=is_zfull(s.tuned, integ, recon))}
    return out


def kernels_of(groups, tuned, integ="vl", recon="plm"):
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
            if k.startswith(st + "_") and k.split("_")[1] in AXES:
                d = AXES.index(k.split("_")[1])
                stage = st if integ == "vl" else ("tracing" if st == "predictor" else "ctucorr")
                other = "cell" if stage == "ctucorr" else "tile"
                xform = "xwarp"
                if integ == "vl" and mask & 16:
                    xform = "xpencil"
                elif integ == "vl" and (mask & 32 if st == "predictor" else (mask & 64 and recon != "ppm")):
                    xform = "xmarch"
                elif integ != "vl" and st == "predictor" and mask & 32 and recon != "ppm":
                    xform = "xmarch"                 # the CTU tracing (the correction keeps its warps)
                name = f"{stage}_{(xform if d == 0 else 'pencil') if mask >> d & 1 else other}"
        ms, cnt = out.get(name, (0.0, 0))
        out[name] = (ms + v, cnt + nl)
    return out


def roofline(prec, groups, steps, n, pk, apk, scheme, tuned=None):
    """Dominant kernel of the step and its achieved fraction of the roofline
    that bounds it.  Algorithmic work per launch: the oracle-counted flops
    and the algorithmic bytes of its units (faces for a sweep, cells for a
    per-cell kernel).  The bound is picked by that arithmetic intensity
    against the ridge (measured FMA peak / measured HBM bandwidth); the other
    side and the kernel's executed flops (ncu counts) are reported beside."""
    integ = scheme[0]
    ks = kernels_of(groups, tuned, integ, scheme[1])
    dom = max(ks, key=lambda k: ks[k][0])
    tot, launches = ks[dom]
    ms = tot / steps
    t_launch = ms / launches * 1e-3
    out = {"kernel": dom, "ms_per_step": ms, "share": tot / sum(groups.values()), "launches": launches,
           "ms_per_launch": ms / launches}
    af = alg_flops(scheme)
    sweep = dom.split("_")[0]
    alu_peak = alu_peak_of(prec, apk)
    yh = is_yhalf(tuned, integ, scheme[1])
    yp = is_yprim(tuned, integ)
    zf = is_zfull(tuned, integ, scheme[1])
    if dom == "corrector_zfull":
        # per cell: one corrector face and the conservative update (the
        # oracle's full-update count, its CT part included)
        bpu = group_bytes(prec, n, integ, False, yh, yp, True)[dom] / n
        fpu = af["per_face"]["corrector"] + af["per_cell"]["full_update"]
        unit_name = "cells"
        tpf = TRAFFIC_PER_FACE.get(dom, {}).get(prec)
        traffic = tpf * n if tpf else None
        executed = None
    elif dom == "predictor_yprim":
        # per cell: its primitives and signal speed and its first-order y face
        bpu = group_bytes(prec, n, integ, False, yh, True, zf)[dom] / n
        fpu = af["per_cell"]["prim_cfl"] + af["per_face"]["predictor"]
        unit_name = "cells"
        tpf = TRAFFIC_PER_FACE.get(dom, {}).get(prec)
        traffic = tpf * n if tpf else None
        executed = None
    elif dom == "corrector_yhalf":
        # per cell: its half-step state and its y face (PLM reconstruction
        # and Riemann solve)
        bpu = group_bytes(prec, n, integ, False, True, yp, zf)[dom] / n
        fpu = af["per_cell"]["half_update"] + af["per_face"]["corrector"]
        unit_name = "cells"
        tpf = TRAFFIC_PER_FACE.get(dom, {}).get(prec)
        traffic = tpf * n if tpf else None
        executed = None
    elif dom == "predictor_fused":
        # per cell: three first-order faces, the three edges, the dt/2 update
        # and the half-step primitives
        bpu = group_bytes(prec, n, integ, True)[dom] / n
        fpu = 3 * af["per_face"]["predictor"] + af["per_cell"]["emf1"] + af["per_cell"]["half_update"]
        unit_name = "cells"
        traffic, executed = None, None
    elif sweep in ("predictor", "corrector", "tracing", "ctucorr"):
        bpu = sweep_bytes_per_face(prec, {"tracing": "tracing", "ctucorr": "ctucorr"}.get(sweep, "vl"))
        fpu = af["per_face"][sweep]
        unit_name = "faces"
        tpf = TRAFFIC_PER_FACE.get(dom, {}).get(prec)
        traffic = tpf * n if tpf else None
        executed = EXEC_FLOPS_PER_FACE.get(sweep) if prec != "fp64" else None
    else:
        stage = dom
        bpu = group_bytes(prec, n, integ, is_fused(tuned, integ), yh, yp, zf)[stage] / launches / n
        fpu = af["per_cell"].get(stage, 0.0)
        unit_name = "cells"
        traffic, executed = None, None
    flops, byts = fpu * n, bpu * n
    ridge = alu_peak * 1e12 / (pk["hbm_gbs"] * 1e9)
    intensity = flops / byts
    ach_tf = flops / t_launch / 1e12
    ach_gbs = byts / t_launch / 1e9
    hbm_view = {"achieved": ach_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach_gbs / pk["hbm_gbs"],
                "algorithmic_bytes_per_launch": byts}
    alu_view = {"achieved": ach_tf, "peak": alu_peak, "unit": "TFLOP/s", "frac": ach_tf / alu_peak,
                "algorithmic_flops_per_launch": flops}
    if intensity > ridge:
        out.update(bound="alu", achieved=ach_tf, peak=alu_peak, unit="TFLOP/s", frac=ach_tf / alu_peak,
                   peak_src=f"{'FP64' if prec == 'fp64' else 'FP32'} FMA peak, {apk['src']}")
    else:
        out.update(bound="hbm", achieved=ach_gbs, peak=pk["hbm_gbs"], unit="GB/s", frac=ach_gbs / pk["hbm_gbs"],
                   peak_src=f"{pk['src']} copy bandwidth (MEASURED_PEAKS.json)")
    out.update(traffic=traffic,
               algorithmic=f"{fpu:.0f} flops (oracle count) and {bpu:.0f} B per {unit_name[:-1]} x {n} {unit_name}"
                           " per launch",
               intensity_flop_per_byte=intensity, ridge_flop_per_byte=ridge, hbm_view=hbm_view, alu_view=alu_view)
    if executed:
        ex_tf = executed * n / t_launch / 1e12
        out["executed_view"] = {"flops_per_face": executed, "achieved": ex_tf, "frac": ex_tf / alu_peak,
                                "intensity_flop_per_byte": executed / bpu,
                                "note": "FADD + FMUL + 2 FFMA per face from ncu; the kernel's identities run "
                                        "fewer operations than the method's count"}
    return out


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _oracle_steps(O, st, scheme, m):
    U, B = st.U.copy(), st.B.copy()
    t0 = time.perf_counter()
    for _ in range(m):
        dt = O.cfl_dt(U, B, st.dx, st.gamma, 0.3)
        O.step(U, B, st.dx, st.gamma, dt, *scheme)
    return time.perf_counter() - t0


def oracle_rate(O, n, scheme, threads, runs, steps):
    """median over `runs` runs of `steps` oracle steps (CFL dt included), after
    one warm-up step, on the n^3 sample of the workload family with
    `threads` OpenMP threads (0: all host threads); cell-updates/s"""
    used = O.set_threads(threads if threads > 0 else (os.cpu_count() or 1))
    st = workload(n)
    _oracle_steps(O, st, scheme, 1)
    rates = [n ** 3 * steps / _oracle_steps(O, st, scheme, steps) for _ in range(runs)]
    O.set_threads(os.cpu_count() or 1)
    return {"value": statistics.median(rates), "runs": runs, "steps": steps, "threads": used,
            "spread": [min(rates), max(rates)]}


def cpu_baseline(scheme):
    """The FP64 oracle as it stands, timed on the host cores on bounded
    samples of the workload family: 64^3 with all host threads (median of
    5 runs of 2 steps) and with 1 thread (median of 3 runs of 1 step), and
    128^3 with all threads (median of 3 runs of 1 step); about 10-20 s of CPU
    work.  The line's value is the all-thread 64^3 rate."""
    from oracle import oracle as O
    allc = oracle_rate(O, 64, scheme, 0, 5, 2)
    one = oracle_rate(O, 64, scheme, 1, 3, 1)
    big = oracle_rate(O, 128, scheme, 0, 3, 1)
    return {"value": allc["value"], "unit": UNIT, "cores": allc["threads"], "kind": "oracle", "cpu": cpu_model(),
            "nproc": os.cpu_count(),
            "sample": f"{'+'.join(scheme)} FP64 oracle steps (CFL dt included) on the ABC workload family "
                      f"(k=4pi, beta=0.5, seed 0): 64^3 all threads, median of 5 runs of 2 steps",
            "one_thread_64": one, "all_threads_64": allc, "all_threads_128": big}


def run_cpu_plan(args):
    """The CPU-baseline plan in full (not a bench line): the FP64 oracle at
    64^3 and 128^3, 1 thread and all host threads, median of 5 runs of 10
    steps after one warm-up step, for VL + PLM + Roe; and the eight
    {VL, CTU} x {PLM, PPM} x {Roe, HLLD} schemes at 64^3 with all threads
    (median of 5 runs of 2 steps)."""
    from oracle import oracle as O
    O.build()
    head = ("vl", "plm", "roe")
    out = {"cpu": cpu_model(), "nproc": os.cpu_count(), "headline": {}, "schemes64_all_threads": {}}
    for n in (64, 128):
        for th in (1, 0):
            key = f"{n}^3/{'1 thread' if th == 1 else 'all threads'}"
            out["headline"][key] = oracle_rate(O, n, head, th, 5, args.cpu_plan_steps)
            print(key, out["headline"][key], flush=True)
    for integ in ("vl", "ctu"):
        for recon in ("plm", "ppm"):
            for riem in ("roe", "hlld"):
                out["schemes64_all_threads"][f"{integ}+{recon}+{riem}"] = oracle_rate(O, 64, (integ, recon, riem),
                                                                                      0, 5, 2)
    print(json.dumps({"mode": "cpu_plan", **out}), flush=True)


def run_features(args):
    """The learned selector's block-feature pass alone (mhd_block_features:
    the primitives, then the 48 features of every 4^3 block) on the n^3
    member of the 384^3 workload's blast family, timed by CUDA events;
    prints one JSON line (not a bench line)."""
    import torch
    from paper_1804_03479_b300 import build as Bld
    Bld.build()
    from paper_1804_03479_b300 import mhd
    from paper_1804_03479_b300 import inputs as I
    n = args.features_n
    st = I.abc_blasts(n, kmult=3, beta=0.1, nblast=10, E=1.0, radius=0.05, seed=2)
    s = mhd.Solver(st.U.shape[1:], st.dx, st.gamma, "vl", "ppm", "hlld", "fp32", 0.3)
    s.set_state(torch.from_numpy(st.U).to("cuda", torch.float32), torch.from_numpy(st.B).to("cuda", torch.float32))
    out = torch.empty((s.nblocks(), 48), dtype=torch.float32, device="cuda")
    for _ in range(max(1, args.warmup)):
        s.block_features(out)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = max(1, min(args.steps, 20))
    e0.record()
    for _ in range(reps):
        s.block_features(out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    s.free()
    print(json.dumps({"mode": "features", "n": n, "blocks": int(out.shape[0]), "reps": reps,
                      "ms_per_pass_with_primitives": ms}), flush=True)


def graph_node_us(torch, stream, nodes=12, reps=200):
    """device time per node of a CUDA graph of `nodes` one-element kernels,
    replayed back to back: the launch gap plus the smallest kernel, an upper
    bound on what each of a graph-replayed step's launches adds"""
    x = torch.zeros(1, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        x.add_(1.0)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(nodes):
                x.add_(1.0)
        for _ in range(10):
            g.replay()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            g.replay()
        e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e3 / (reps * nodes)


def batch_variant(torch, mhd, K, stream, pk, apk):
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
    mask = s.sweep_pencils()[0]
    nl = s.launches_per_step()
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
    nl_loop = ctxs[0].launches_per_step()
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
    node_us = graph_node_us(torch, stream)
    return {"value": ncell / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": K, "boxes": 48,
            "graph_launch_cost": {"us_per_node_upper_bound": node_us,
                                  "ms_per_step_upper_bound": nl * node_us * 1e-3,
                                  "frac_of_step_upper_bound": nl * node_us * 1e-3 / ms,
                                  "how": "12-node graph of one-element kernels replayed back to back"},
            "step_roofline": step_roofline("fp32", ncell, ms, pk, apk, ("vl", "ppm", "hlld"),
                                           fused=bool(mask & 8)),
            "cells": ncell, "sides": sides, "scheme": "vl+ppm+hlld", "precision": "fp32",
            "sweep_tiling": {"tile_len": tl, "blocks_per_sm": bps, "autotune_ms_per_step": tune_ms},
            "pencil_mask": mask, "launches_per_step": nl, "graph": True,
            "per_box_loop": {"value": ncell / (ms_loop * 1e-3), "ms_per_step": ms_loop,
                             "launches_per_step": nl_loop * 48},
            "speedup_vs_per_box_loop": ms_loop / ms}


def learned_variant(torch, mhd, K, stream, pk, apk):
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
    for name in ("full", "selected", "cheap"):
        s = mhd.Solver(st.U.shape[1:], st.dx, st.gamma, *(LRN.CHEAP if name == "cheap" else LRN.FULL), "fp32",
                       0.3, stream=stream.cuda_stream, pfloor=LRN.PFLOOR)
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
        if name != "selected":            # the plain schemes' own sweep configuration
            groups = fold_groups(groups, {"pencil_mask": s.sweep_pencils()[0]}, "vl",
                                 (LRN.CHEAP if name == "cheap" else LRN.FULL)[1], LRN.PFLOOR)
        if name == "selected":
            out["cheap_fraction_blocks"], out["cheap_fraction_tiles"] = s.selector_stats()
        s.get_state(U, B)
        states[name] = (U, B)
        out[name] = {"value": st.U[0].size / (ms * 1e-3), "ms_per_step": ms,
                     "kernel_ms_per_step": {k: v / rec for k, v in stages_of(groups).items()},
                     "sweep_ms_per_step": {k: v / rec for k, v in groups.items()
                                           if "_" in k and k.split("_")[1] in AXES},
                     "floored_cell_steps": s.floor_count()}
        s.free()
    net.free()
    names = ["rho", "Mx", "My", "Mz", "e", "Bx", "By", "Bz"]
    l1 = LRN.rel_l1_fields(states["selected"], states["full"])
    l1c = LRN.rel_l1_fields(states["cheap"], states["full"])
    ncell = st.U[0].size
    # algorithmic flops of the selected step: the cheap and full schemes in
    # the proportion of sweep units each ran, plus the network (2 layers of
    # 48x64 and 64x64 multiply-adds per 4^3 block)
    fc = out["cheap_fraction_tiles"]
    mlp = 2.0 * (48 * 64 + 64 * 64 + 64) / 64.0
    fl_sel = fc * alg_flops(LRN.CHEAP)["total"] + (1 - fc) * alg_flops(LRN.FULL)["total"] + mlp
    return {"value": out["selected"]["value"], "unit": UNIT, "ms_per_step": out["selected"]["ms_per_step"],
            "steps": K, "workload": "abc384_k6pi_beta0.1 + 10 blasts (E=1, r<0.05, seed 2)",
            "precision": "fp32", "full_path": out["full"], "selected_path": out["selected"],
            "cheap_path": out["cheap"],
            "step_roofline": step_roofline("fp32", ncell, out["selected"]["ms_per_step"], pk, apk, LRN.FULL,
                                           flops_per_cell=fl_sel),
            "speedup_vs_all_full": out["full"]["ms_per_step"] / out["selected"]["ms_per_step"],
            "speedup_of_all_cheap_vs_all_full": out["full"]["ms_per_step"] / out["cheap"]["ms_per_step"],
            "cheap_fraction_blocks": out["cheap_fraction_blocks"], "cheap_fraction_tiles": out["cheap_fraction_tiles"],
            "rel_l1_vs_all_full_after_steps": dict(zip(names, l1)),
            "all_cheap_rel_l1_vs_all_full_after_steps": dict(zip(names, l1c)),
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
    ap.add_argument("--variants", default="fp64,mixed",
                    help="other precisions measured beside the main line (comma list; none: no others)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-matrix", action="store_true", help="skip the 16 scheme x precision combinations")
    ap.add_argument("--matrix-steps", type=int, default=100, help="FP32 steps per scheme (FP64: a tenth)")
    ap.add_argument("--no-autotune", action="store_true", help="default sweep tiling instead of the autotuned one")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--stress", action="store_true", help="mixed-precision stress run (not a bench line)")
    ap.add_argument("--stress-steps", type=int, default=500)
    ap.add_argument("--stress-shape", type=int, nargs=3, default=[512, 256, 256])
    ap.add_argument("--stress-pfloor", type=float, default=1e-5)
    ap.add_argument("--cpu-plan", action="store_true", help="the full CPU-baseline plan (not a bench line)")
    ap.add_argument("--cpu-plan-steps", type=int, default=10)
    ap.add_argument("--pencil-mask", type=int, default=None,
                    help="sweep forms of the main line (mhd_set_sweep_pencils), after any autotuning")
    ap.add_argument("--pencil-len", type=int, default=None)
    ap.add_argument("--emf-staging", type=int, default=None, choices=[0, 1, 2],
                    help="edge-field form of the main line (mhd_set_emf_staging)")
    ap.add_argument("--features-n", type=int, default=None,
                    help="time only the learned selector's block-feature pass on the n^3 blast state "
                         "(not a bench line)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.stress:
        return run_stress(args)
    if args.cpu_plan:
        return run_cpu_plan(args)
    if args.features_n:
        return run_features(args)

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
    apk = alu_peaks(mhd)
    scheme = (args.integrator, args.recon, args.riemann)
    st = workload(args.n)
    n = args.n ** 3
    stream = torch.cuda.Stream()
    clk = Clocks(local)
    clk.start()
    ms, groups, rec, s = time_variant(torch, mhd, st, args.precision, scheme, args.steps, args.warmup, dist, stream,
                                      tune=not args.no_autotune,
                                      forms=(args.pencil_mask, args.pencil_len, args.emf_staging))
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
        "roofline": roofline(args.precision, groups, rec, n, pk, apk, scheme, s.tuned) if rec else None,
        "step_roofline": step_roofline(args.precision, n, ms / args.steps, pk, apk, scheme,
                                       fused=is_fused(s.tuned, scheme[0]),
                                       yhalf=is_yhalf(s.tuned, scheme[0], scheme[1]),
                                       yprim=is_yprim(s.tuned, scheme[0]),
                                       zfull=is_zfull(s.tuned, scheme[0], scheme[1])),
        "alu_peaks_tflops": apk,
        "kernel_ms_per_step": {k: v / rec for k, v in stages_of(groups).items()} if rec else None,
        "sweep_ms_per_step": {k: v / rec for k, v in groups.items() if "_" in k and k.split("_")[1] in AXES}
        if rec else None,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rank == 0:
        variants = {}
        for prec in [p for p in args.variants.split(",") if p in SIZES and p != args.precision]:
            kv = max(3, min(args.steps, 10))
            msv, gv, recv, sv = time_variant(torch, mhd, st, prec, scheme, kv, 2, None, stream,
                                             tune=not args.no_autotune)
            sv.free()
            vv = n * kv / (msv * 1e-3)
            variants[prec] = {"value": vv, "unit": UNIT, "ms_per_step": msv / kv, "steps": kv,
                              "vs_p100_paper": vv / PAPER_P100[prec] if prec in PAPER_P100 else None,
                              "roofline": roofline(prec, gv, recv, n, pk, apk, scheme, sv.tuned)
                              if recv else None,
                              "step_roofline": step_roofline(prec, n, msv / kv, pk, apk, scheme,
                                                             fused=is_fused(sv.tuned, scheme[0]),
                                                             yhalf=is_yhalf(sv.tuned, scheme[0], scheme[1]),
                                                             yprim=is_yprim(sv.tuned, scheme[0]),
                                                             zfull=is_zfull(sv.tuned, scheme[0], scheme[1])),
                              "kernel_ms_per_step": {k: v / recv for k, v in stages_of(gv).items()} if recv else None,
                              "sweep": sv.tuned}
        if not args.no_matrix:
            variants["schemes256"] = scheme_matrix(torch, mhd, st, args.matrix_steps, max(2, args.matrix_steps // 10),
                                                   stream, pk, apk)
        if not args.no_batch:
            variants["batch48"] = batch_variant(torch, mhd, max(3, min(args.steps, 10)), stream, pk, apk)
        if not args.no_learned:
            variants["learned384"] = learned_variant(torch, mhd, max(3, min(args.steps, 10)), stream, pk, apk)
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
