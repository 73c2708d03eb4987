"""The benchmark's host logic on CPU: the reference arm (the oracle timed on
the host) prints the contract's JSON line, and the roofline picks the
dominant kernel from the per-group times and computes its fraction from the
flops per face and the event time."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_the_contract_line():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 2
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["metric"] == json.load(open(os.path.join(ROOT, "BASELINE.json")))["metric"]


def test_roofline_of_the_dominant_kernel():
    import bench
    n = 256 ** 3
    steps = 10
    # per-group totals over 10 steps (ms): the y and z corrector pencils dominate
    groups = {"prim_cfl": 2.3, "predictor_x": 4.8, "predictor_y": 3.0, "predictor_z": 3.0, "emf1": 3.0,
              "half_update": 5.0, "corrector_x": 6.2, "corrector_y": 4.9, "corrector_z": 4.9, "emf2": 3.0,
              "full_update": 4.8}
    tuned = {"pencil_mask": 7}
    ks = bench.kernels_of(groups, tuned)
    assert ks["corrector_pencil"] == (9.8, 2) and ks["corrector_xwarp"] == (6.2, 1)
    pk = {"hbm_gbs": 6491.2, "src": "measured"}
    apk = {"fp32": 70.0, "fp64": 1.2, "src": "test"}
    scheme = ("vl", "plm", "roe")
    r = bench.roofline("fp32", groups, steps, n, pk, apk, scheme, tuned)
    assert r["kernel"] == "corrector_pencil" and r["launches"] == 2
    per_launch_s = 9.8 / steps / 2 * 1e-3
    fpf = bench.alg_flops(scheme)["per_face"]["corrector"]
    # the oracle's nontrivial operations: one reconstruction and one Roe solve per face
    assert 1200 < fpf < 2500
    flops, byts = n * fpf, n * bench.sweep_bytes_per_face("fp32")
    assert r["intensity_flop_per_byte"] == pytest.approx(flops / byts)
    assert r["ridge_flop_per_byte"] == pytest.approx(70.0e12 / 6491.2e9)
    # above the ridge: the arithmetic side binds
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["peak"] == 70.0
    assert r["achieved"] == pytest.approx(flops / per_launch_s / 1e12, rel=1e-12)
    assert r["frac"] == pytest.approx(r["achieved"] / 70.0, rel=1e-12)
    assert r["hbm_view"]["frac"] == pytest.approx(byts / per_launch_s / 6491.2e9, rel=1e-12)
    ex = r["executed_view"]
    assert ex["achieved"] == pytest.approx(n * bench.EXEC_FLOPS_PER_FACE["corrector"] / per_launch_s / 1e12)
    tpf = bench.TRAFFIC_PER_FACE.get("corrector_pencil", {}).get("fp32")
    assert r["traffic"] == (pytest.approx(tpf * n) if tpf else None)
    # with a much faster arithmetic pipe the same kernel is HBM-bound
    r2 = bench.roofline("fp32", groups, steps, n, pk, {"fp32": 1e4, "fp64": 1.0, "src": "t"}, scheme, tuned)
    assert r2["bound"] == "hbm" and r2["frac"] == pytest.approx(r["hbm_view"]["frac"])
    # without pencils the same groups belong to the tile kernels
    assert "corrector_tile" in bench.kernels_of(groups, {"pencil_mask": 0})
    # x by aligned marching warps: bit 5 the predictor, bit 6 the PLM corrector
    ks = bench.kernels_of(groups, {"pencil_mask": 103})
    assert ks["predictor_xmarch"] == (4.8, 1) and ks["corrector_xmarch"] == (6.2, 1)
    ks = bench.kernels_of(groups, {"pencil_mask": 103}, "vl", "ppm")
    assert ks["predictor_xmarch"] == (4.8, 1) and ks["corrector_xwarp"] == (6.2, 1)
    ks = bench.kernels_of(groups, {"pencil_mask": 39})
    assert ks["predictor_xmarch"] == (4.8, 1) and ks["corrector_xwarp"] == (6.2, 1)
    ks = bench.kernels_of(groups, {"pencil_mask": 119})          # bit 4 takes precedence
    assert ks["predictor_xpencil"] == (4.8, 1) and ks["corrector_xpencil"] == (6.2, 1)
    ks = bench.kernels_of(groups, {"pencil_mask": 39}, "ctu")    # CTU: the x tracing marches
    assert ks["tracing_xmarch"] == (4.8, 1) and ks["ctucorr_xwarp"] == (6.2, 1)
    ks = bench.kernels_of(groups, {"pencil_mask": 39}, "ctu", "ppm")
    assert ks["tracing_xwarp"] == (4.8, 1) and ks["ctucorr_xwarp"] == (6.2, 1)


def test_roofline_of_a_ctu_step():
    """CTU's stages are the tracing sweeps and the transverse corrections:
    their own kernel names, flop counts and algorithmic bytes"""
    import bench
    n = 256 ** 3
    steps = 10
    groups = {"prim_cfl": 2.3, "predictor_x": 8.1, "predictor_y": 6.7, "predictor_z": 7.2, "emf1": 3.0,
              "half_update": 5.0, "corrector_x": 6.4, "corrector_y": 5.9, "corrector_z": 5.8, "emf2": 3.0,
              "full_update": 4.8}
    tuned = {"pencil_mask": 7}
    ks = bench.kernels_of(groups, tuned, "ctu")
    assert ks["tracing_pencil"] == (pytest.approx(13.9), 2) and ks["tracing_xwarp"] == (8.1, 1)
    assert ks["ctucorr_pencil"] == (pytest.approx(11.7), 2) and ks["ctucorr_xwarp"] == (6.4, 1)
    assert "ctucorr_cell" in bench.kernels_of(groups, {"pencil_mask": 6}, "ctu")
    pk = {"hbm_gbs": 6491.2, "src": "measured"}
    apk = {"fp32": 70.0, "fp64": 1.2, "src": "test"}
    scheme = ("ctu", "plm", "roe")
    r = bench.roofline("fp32", groups, steps, n, pk, apk, scheme, tuned)
    assert r["kernel"] == "tracing_pencil"
    fpf = bench.alg_flops(scheme)["per_face"]["tracing"]
    want = n * fpf / (13.9 / steps / 2 * 1e-3) / 1e12
    assert r["alu_view"]["achieved"] == pytest.approx(want, rel=1e-12)
    # tracing: W (8) and B_n in, the flux and both traced states (21) out
    assert bench.sweep_bytes_per_face("fp32", "tracing") == 4 * (8 + 1 + 21)
    assert r["hbm_view"]["algorithmic_bytes_per_launch"] == n * 4 * 30
    assert bench.group_bytes("fp32", n, "ctu")["corrector_sweeps"] == 3 * n * 4 * 37


def test_step_roofline_binds_at_the_lower_ceiling():
    import bench
    n = 256 ** 3
    pk = {"hbm_gbs": 6491.2, "src": "measured"}
    apk = {"fp32": 70.0, "fp64": 1.2, "src": "test"}
    scheme = ("vl", "plm", "roe")
    r = bench.step_roofline("fp32", n, 4.4, pk, apk, scheme)
    cups = n / 4.4e-3
    fl = bench.alg_flops(scheme)["total"]
    assert r["hbm"]["ceiling_cell_updates_per_s"] == pytest.approx(6491.2e9 / 64)
    assert r["alu"]["ceiling_cell_updates_per_s"] == pytest.approx(70e12 / fl)
    assert r["bound"] == "alu" and r["frac"] == pytest.approx(cups / (70e12 / fl))
    r64 = bench.step_roofline("fp64", n, 150.0, pk, apk, scheme)
    assert r64["bound"] == "alu" and r64["alu"]["peak_tflops"] == 1.2
    rm = bench.step_roofline("mixed", n, 6.0, pk, apk, scheme)
    assert rm["hbm"]["bytes_per_cell_update"] == 96 and rm["alu"]["peak_tflops"] == 70.0


def test_roofline_of_the_y_corrector_with_the_half_update():
    """pencil-mask bit 7 (with bit 1, PLM, no bit 3): the library's half
    group times the y corrector that forms the half-step states and its y
    group is empty; the bench names them corrector_yhalf, whose work per cell
    is the half update's plus one corrector face"""
    import bench
    n = 256 ** 3
    steps = 10
    groups = {"prim_cfl": 1.8, "predictor_x": 2.7, "predictor_y": 2.7, "predictor_z": 2.7, "emf1": 2.9,
              "half_update": 7.1, "corrector_x": 5.1, "corrector_y": 0.01, "corrector_z": 4.7, "emf2": 3.0,
              "full_update": 4.1}
    tuned = {"pencil_mask": 231}
    assert bench.is_yhalf(tuned) and bench.is_yhalf(tuned, "vl", "ppm") and not bench.is_yhalf(tuned, "ctu")
    assert not bench.is_yhalf({"pencil_mask": 103}) and not bench.is_yhalf({"pencil_mask": 239})
    g = bench.fold_groups(groups, tuned, "vl", "plm")
    assert "half_update" not in g and "corrector_y" not in g
    assert g["corrector_yhalf"] == pytest.approx(7.11)
    assert bench.fold_groups(groups, tuned, "vl", "ppm") == g
    st = bench.stages_of(g)
    assert st["corrector_yhalf"] == pytest.approx(7.11) and st["corrector_sweeps"] == pytest.approx(9.8)
    pk = {"hbm_gbs": 6491.2, "src": "measured"}
    apk = {"fp32": 75.0, "fp64": 1.0, "src": "test"}
    scheme = ("vl", "plm", "roe")
    r = bench.roofline("fp32", g, steps, n, pk, apk, scheme, tuned)
    assert r["kernel"] == "corrector_yhalf" and r["launches"] == 1
    af = bench.alg_flops(scheme)
    fpu = af["per_cell"]["half_update"] + af["per_face"]["corrector"]
    assert r["alu_view"]["achieved"] == pytest.approx(n * fpu / (7.11 / steps * 1e-3) / 1e12, rel=1e-12)
    # bytes: rho, M, e and the faces (32), the 15 fluxes and 3 edge fields
    # (72) in; the half-step faces (12), primitives (32) and y fluxes (28) out
    assert r["hbm_view"]["algorithmic_bytes_per_launch"] == n * (32 + 72 + 12 + 32 + 28)
    gb = bench.group_bytes("fp32", n, "vl", False, True)
    assert "half_update" not in gb and gb["corrector_sweeps"] == 2 * n * 64
    assert sum(gb.values()) == sum(bench.group_bytes("fp32", n, "vl").values()) - n * 64 + n * 28


def test_folding_of_the_y_predictor_with_the_primitives():
    """pencil-mask bit 8 (with bit 1, no bit 3, no pressure floor): the
    primitive group times the y predictor that forms the primitives and the
    y predictor group is empty; with bit 7 as well both fold"""
    import bench
    n = 256 ** 3
    groups = {"prim_cfl": 7.2, "predictor_x": 2.7, "predictor_y": 0.01, "predictor_z": 2.7, "emf1": 2.9,
              "half_update": 19.0, "corrector_x": 5.1, "corrector_y": 0.01, "corrector_z": 4.7, "emf2": 3.0,
              "full_update": 5.7}
    assert bench.is_yprim({"pencil_mask": 487}) and not bench.is_yprim({"pencil_mask": 487}, "vl", 1e-4)
    assert not bench.is_yprim({"pencil_mask": 231}) and not bench.is_yprim({"pencil_mask": 487}, "ctu")
    g = bench.fold_groups(groups, {"pencil_mask": 487}, "vl", "plm")
    assert set(g) == {"predictor_yprim", "predictor_x", "predictor_z", "emf1", "corrector_yhalf", "corrector_x",
                      "corrector_z", "emf2", "full_update"}
    assert g["predictor_yprim"] == pytest.approx(7.21) and g["corrector_yhalf"] == pytest.approx(19.01)
    g2 = bench.fold_groups(groups, {"pencil_mask": 359}, "vl", "ppm")
    assert "predictor_yprim" in g2 and "half_update" in g2 and "corrector_y" in g2
    g3 = bench.fold_groups(groups, {"pencil_mask": 487}, "vl", "ppm")
    assert "predictor_yprim" in g3 and "corrector_yhalf" in g3 and "corrector_z" in g3
    r = bench.roofline("mixed", g, 10, n, {"hbm_gbs": 6491.2, "src": "measured"},
                       {"fp32": 75.0, "fp64": 1.0, "src": "test"}, ("vl", "plm", "roe"), {"pencil_mask": 487})
    assert r["kernel"] == "corrector_yhalf"
    gb = bench.group_bytes("mixed", n, "vl", False, True, True)
    szu, sze, szr = bench.SIZES["mixed"]
    assert gb["predictor_yprim"] == n * (4 * szu + 4 * sze + 8 * szr + 7 * szr)
    assert gb["predictor_sweeps"] == 2 * n * bench.sweep_bytes_per_face("mixed", "vl")


def test_folding_of_the_z_corrector_with_the_conservative_update():
    """pencil-mask bit 9 (with bit 2, PLM, no bit 3): the z corrector group
    is corrector_zfull and the full-update group times CT alone"""
    import bench
    n = 256 ** 3
    groups = {"prim_cfl": 1.8, "predictor_x": 2.7, "predictor_y": 2.7, "predictor_z": 2.7, "emf1": 2.9,
              "half_update": 7.1, "corrector_x": 5.1, "corrector_y": 0.01, "corrector_z": 6.9, "emf2": 3.0,
              "full_update": 1.0}
    tuned = {"pencil_mask": 743}
    assert bench.is_zfull(tuned) and not bench.is_zfull(tuned, "vl", "ppm") and not bench.is_zfull({"pencil_mask": 231})
    g = bench.fold_groups(groups, tuned, "vl", "plm")
    assert g["corrector_zfull"] == 6.9 and "corrector_z" not in g and g["corrector_yhalf"] == pytest.approx(7.11)
    ks = bench.kernels_of(g, tuned)
    assert ks["corrector_zfull"] == (6.9, 1) and ks["corrector_xmarch"] == (5.1, 1)
    gb = bench.group_bytes("fp32", n, "vl", False, True, False, True)
    assert gb["corrector_zfull"] == n * 4 * (9 + 3 + 10 + 10)     # W, B_n; F_z 3; rho, M, e in and out; F_x, F_y
    assert gb["full_update"] == n * 4 * 9 and gb["corrector_sweeps"] == n * 64
    r = bench.roofline("fp32", g, 10, n, {"hbm_gbs": 6491.2, "src": "measured"},
                       {"fp32": 75.0, "fp64": 1.0, "src": "test"}, ("vl", "plm", "roe"), tuned)
    assert r["kernel"] == "corrector_yhalf"
