"""The multi-rank logic of bench.py on CPU with the gloo backend (world size
2): every rank advances its own replica (the path has no exchange step), the
job's time is the slowest rank's and the value aggregates all ranks' cells."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import oracle as O
    from paper_1804_03479_b300 import inputs as I
    # each rank: one replica of a small box, advanced by the CPU reference,
    # a deliberately different amount of work per rank
    st = I.abc(8, kmult=1, seed=rank)
    U, B = st.U.copy(), st.B.copy()
    for _ in range(1 + rank):
        O.step(U, B, st.dx, st.gamma, O.cfl_dt(U, B, st.dx, st.gamma, 0.3))
    ms_local = 10.0 * (rank + 1)
    ms = bench.max_over_ranks(torch, ms_local, dist, "cpu")
    v = bench.aggregate_value(world, 512, 3, ms)
    ws, r, _ = bench.dist_info()
    out[rank] = (ms, v, ws, r, float(U[0].sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for rank, (ms, v, ws, r, mass) in res.items():
        assert ms == 20.0                      # the slowest rank's time on every rank
        assert v == 2 * 512 * 3 / 20e-3        # all ranks' cell-updates over that time
        assert ws == 2 and r == rank
        assert abs(mass - 512.0) < 1e-9        # each replica conserves its own mass
