"""Multi-rank plumbing of bench.py on CPU: two gloo ranks (world size 2).

bench.py shards the workload as independent replicas (one system per rank,
no collective on the data path); the only collectives are the barrier around
the timed region and the max-over-ranks reduction of the elapsed time.  This
runs both with the gloo backend, as torchrun would launch them.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    ws, r, local = bench.dist_setup()
    try:
        bench.barrier(ws)
        t = bench.max_over_ranks(1.5 + r, ws, "cpu")   # rank r "took" 1.5 + r seconds
        bench.barrier(ws)
        out.put((r, ws, local, dist.get_backend(), t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_barrier_and_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [x[0] for x in res] == [0, 1]
    for r, ws, local, backend, t in res:
        assert ws == 2 and local == r and backend == "gloo"
        assert t == 2.5          # every rank reports the slowest rank's time


def test_single_rank_helpers_are_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25
    bench.barrier(1)
