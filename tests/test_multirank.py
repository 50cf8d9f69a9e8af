"""The N > 1 path of bench.py on CPU: two gloo ranks, replicas only (no data
collective), timing is the max over ranks and units are summed."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    from paper_1807_07914_gb300 import inputs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_setup()
    t = bench.reduce_max(1.5 + rank, ws)
    units = bench.reduce_sum(304, ws)
    th = inputs.thetas(4, 8, inputs.rng_for(5, 100 + r))
    q.put((r, t, units, float(th[0, 0])))
    dist.destroy_process_group()


def test_two_rank_timing_and_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.5, 2.5]          # max over ranks
    assert [r[2] for r in res] == [608.0, 608.0]      # whole-job units
    assert res[0][3] != res[1][3]                     # each rank its own theta rows
