"""Operation counts of the oracle's step (``flopcount.cpp``): the algorithmic
work of the method per cell-update, per stage, for a scheme combination.

TEST AND MEASUREMENT INFRASTRUCTURE ONLY: used by ``tests/`` and by the
benchmark's roofline numerator; the product path never imports it.

The counting build is the oracle's own C source compiled as C++ with a
scalar type that counts additions (and subtractions), multiplications,
divisions, square roots, comparisons and absolute values.  A "flop" here is
one addition, multiplication, division or square root (each counted once);
comparisons and absolute values are reported beside them, not in the flops.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flopcount.cpp")
_ORC = os.path.join(_HERE, "mhd_oracle.c")
_LIB = os.path.join(_HERE, "libmhd_flopcount.so")

KINDS = ("add", "mul", "div", "sqrt", "cmp", "abs", "add0", "mul0")
FLOP_KINDS = ("add", "mul", "div", "sqrt")

_lib = None


def build(force: bool = False) -> str:
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_ORC))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        cmd = ["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-w", "-shared", "-fPIC",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True, cwd=_HERE)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ll = ctypes.POINTER(ctypes.c_longlong)
        L.fc_reset.restype = None
        L.fc_mark.argtypes = [ctypes.c_char_p]
        L.fc_mark.restype = None
        L.fc_totals.argtypes = [ll]
        L.fc_totals.restype = None
        L.fc_nstages.restype = ctypes.c_int
        L.fc_stage.argtypes = [ctypes.c_int, ctypes.c_char_p, ctypes.c_int, ll]
        L.fc_stage.restype = None
        L.orc_step_full.restype = ctypes.c_long
        L.orc_step_full.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [ctypes.c_int] * 3 + \
                                   [ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp, ctypes.POINTER(ctypes.c_long)]
        L.orc_cfl_dt_full.restype = ctypes.c_double
        L.orc_cfl_dt_full.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 4 + [ctypes.c_int, dp, dp]
        _lib = L
    return _lib


def _p(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _counts(getter):
    out = (ctypes.c_longlong * 8)()
    getter(out)
    return dict(zip(KINDS, (int(x) for x in out)))


def count_step(U, B, dx, gamma, dt, integrator, recon, riemann, cfl=0.3, advance=True):
    """Count one step (the CFL dt reduction included, as the step's first
    stage "cfl") on the state U, B (advanced in place if `advance`).
    Returns {stage: {kind: count}} with the totals under "total", all per
    cell-update (divided by the number of cells)."""
    from oracle.oracle import INTEGRATORS, RECONS, SOLVERS
    L = lib()
    if not advance:
        U, B = U.copy(), B.copy()
    nz, ny, nx = U.shape[1:]
    n = nx * ny * nz
    L.fc_reset()
    L.orc_cfl_dt_full(nx, ny, nz, dx, gamma, cfl, 0.0, 0, _p(U), _p(B))
    L.fc_mark(b"cfl")
    nfl = ctypes.c_long(0)
    L.orc_step_full(nx, ny, nz, dx, gamma, INTEGRATORS[integrator], RECONS[recon], SOLVERS[riemann], dt,
                    0.0, 0, _p(U), _p(B), ctypes.byref(nfl))
    out = {}
    buf = ctypes.create_string_buffer(64)
    for i in range(L.fc_nstages()):
        c = (ctypes.c_longlong * 8)()
        L.fc_stage(i, buf, 64, c)
        out[buf.value.decode()] = {k: int(v) / n for k, v in zip(KINDS, c)}
    out["total"] = {k: v / n for k, v in _counts(L.fc_totals).items()}
    return out


def flops(c):
    """flops of one count dict: add + mul + div + sqrt"""
    return sum(c[k] for k in FLOP_KINDS)


# the workload the stored table is counted on: the 256^3 benchmark's initial
# state family (ABC field, beta = 0.5, seed 0) at 32^3 with 32 cells per
# wavelength; counts of the smooth parts do not depend on the state, the
# limiter and solver branches by about 2 % between 16^3 and 32^3
TABLE_STATE = dict(n=32, kmult=1, beta=0.5, seed=0)
TABLE = os.path.join(_HERE, "flops_per_cell.json")
COMBOS = [(i, r, s) for i in ("vl", "ctu") for r in ("plm", "ppm") for s in ("roe", "hlld", "hlle")] + \
         [("vl", "plm_prim", "hlle"), ("vl", "plm_prim", "roe")]


def count_combo(integrator, recon, riemann, state=TABLE_STATE):
    """per-stage counts per cell-update of one step of a combination on the
    table's state; every count dict gains "flops" (add + mul + div + sqrt)
    and "nontrivial" (flops minus the additions of a zero and the
    multiplications by 0 or +-1)"""
    from oracle import oracle as O
    from paper_1804_03479_b300 import inputs as I
    st = I.abc(state["n"], kmult=state["kmult"], beta=state["beta"], seed=state["seed"])
    dt = O.cfl_dt(st.U, st.B, st.dx, st.gamma, 0.3)
    c = count_step(st.U.copy(), st.B.copy(), st.dx, st.gamma, dt, integrator, recon, riemann)
    for v in c.values():
        v["flops"] = flops(v)
        v["nontrivial"] = v["flops"] - v["add0"] - v["mul0"]
    return c


def write_table(path=TABLE):
    """Write the per-combination, per-stage counts (per cell-update) as JSON."""
    import json
    out = {"state": TABLE_STATE, "unit": "operations per cell-update", "combos": {}}
    for combo in COMBOS:
        out["combos"]["-".join(combo)] = count_combo(*combo)
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
    return path


if __name__ == "__main__":
    print(write_table())
