"""The multi-rank path of bench.py on CPU: world_size 2 over gloo.  Each rank
is an independent replica (no data-path collective); the ranks meet only at
the barrier around the timed region and in the max-reduction of its time,
and the reported value is the units of all ranks over that max."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp


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
    w, r, local = bench.dist_env()
    d = bench.Dist(w, r, "gloo")
    d.barrier()
    t = d.max(10.0 + 5.0 * rank)          # rank 1 is the slow one
    units = 100 * w                       # every rank processed 100 units
    q.put((rank, w, local, t, units / t))
    d.close()


def test_two_replicas_max_time_and_aggregate_value():
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
    for rank, world, local, t, value in res:
        assert world == 2 and local == rank
        assert t == 15.0                   # max over ranks
        assert abs(value - 200 / 15.0) < 1e-12
