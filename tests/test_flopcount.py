"""The operation-counting build of the oracle (oracle/flopcount.cpp) and the
stored table of algorithmic operations per cell-update it writes
(oracle/flops_per_cell.json), which the benchmark's roofline reads.

- The counting build runs the oracle's own source: its step gives the
  oracle's state bit for bit, so what it counts is what the oracle computes.
- The stage counts add up to the total.
- Stages that do not involve the Riemann solver or the reconstruction
  (the CFL reduction, the primitives, the edge fields, the updates) count the
  same for every solver.
- The counter itself: one physical flux of Eq. 7 written out has a known
  number of operations.
- The stored table is what the counting build gives now (it cannot go stale).
"""
import json

import numpy as np
import pytest

from oracle import flops as FL
from oracle import oracle as orc
from paper_1804_03479_b300 import inputs as I


@pytest.mark.parametrize("combo", [("vl", "plm", "roe"), ("ctu", "ppm", "hlld"), ("vl", "plm_prim", "hlle")])
def test_counting_build_is_the_oracle(combo):
    st = I.abc(12, kmult=1, beta=0.5, seed=4, noise=1e-2)
    dt = orc.cfl_dt(st.U, st.B, st.dx, st.gamma, 0.3)
    U1, B1 = st.U.copy(), st.B.copy()
    c = FL.count_step(U1, B1, st.dx, st.gamma, dt, *combo)
    U2, B2 = st.U.copy(), st.B.copy()
    orc.step(U2, B2, st.dx, st.gamma, dt, *combo)
    assert np.array_equal(U1, U2) and np.array_equal(B1, B2)
    stages = {k: v for k, v in c.items() if k != "total"}
    for kind in FL.KINDS:
        assert abs(sum(v[kind] for v in stages.values()) - c["total"][kind]) <= 1e-9 * (1 + c["total"][kind])
    assert FL.flops(c["total"]) > 1000


def test_solver_independent_stages_count_alike():
    st = I.abc(12, kmult=1, beta=0.5, seed=4)
    dt = orc.cfl_dt(st.U, st.B, st.dx, st.gamma, 0.3)
    ref = None
    for solver in ("roe", "hlld", "hlle"):
        c = FL.count_step(st.U.copy(), st.B.copy(), st.dx, st.gamma, dt, "vl", "plm", solver)
        row = [FL.flops(c[s]) for s in ("cfl", "edge_emf", "half_update", "full_update")]
        if ref is None:
            ref = row
        assert row == ref, solver


def test_counter_on_a_known_formula():
    """The CFL stage per cell: the 8 primitives need 3 divisions (velocities)
    and the pressure; then per axis one fast speed with a square root of the
    discriminant and one of c_f^2 -- 6 square roots per cell in all."""
    st = I.abc(8, kmult=1, beta=0.5, seed=1)
    dt = orc.cfl_dt(st.U, st.B, st.dx, st.gamma, 0.3)
    c = FL.count_step(st.U.copy(), st.B.copy(), st.dx, st.gamma, dt, "vl", "plm", "hlle")
    assert c["cfl"]["sqrt"] == 6.0
    assert c["cfl"]["div"] >= 3.0


def test_stored_table_is_current():
    with open(FL.TABLE) as fh:
        table = json.load(fh)
    assert table["state"] == FL.TABLE_STATE
    assert set(table["combos"]) == {"-".join(c) for c in FL.COMBOS}
    for combo in [("vl", "plm", "roe"), ("ctu", "plm", "hlld")]:
        fresh = FL.count_combo(*combo)
        stored = table["combos"]["-".join(combo)]
        for stage, v in fresh.items():
            for kind in ("flops", "nontrivial", "sqrt", "div"):
                assert stored[stage][kind] == pytest.approx(v[kind], rel=1e-12), (combo, stage, kind)
