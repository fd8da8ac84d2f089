"""The benchmark's multi-process logic on CPU: two gloo ranks join through the same
environment torchrun sets, time-like values are max-reduced over the ranks, the barrier
holds both, and the records of all ranks add up (weak scaling: each rank its own hour)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "GNM_BENCH_BACKEND": "gloo"})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup(world)
    assert (w, r, local) == (world, rank, rank)
    t = 10.0 * (rank + 1)  # rank 1 is the slow one
    bench.barrier(w)
    worst = bench.max_over_ranks(t, w)
    records = bench.max_over_ranks(-1.0, w)  # max of equal values is the value
    out.put((rank, worst, records))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    codes = [p.exitcode for p in procs]
    assert codes == [0, 0], codes
    got = sorted(q.get(timeout=5) for _ in range(world))
    assert [g[1] for g in got] == [20.0, 20.0]  # every rank sees the slowest rank's time
    assert [g[2] for g in got] == [-1.0, -1.0]
