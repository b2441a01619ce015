"""The N>1 host path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Each GPU runs independent instances (weak scaling, no data-path collective);
the ranks only meet for a barrier around the timed region and for the
max (time) / sum (work) reductions that give the whole-job value.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    ws, r, local = bench.dist_setup()
    bench.barrier(ws)
    t = bench.max_over_ranks(ws, 1.0 + rank)            # slowest rank sets the time
    w = bench.sum_over_ranks(ws, 10.0 * (rank + 1))     # work of all ranks
    bench.barrier(ws)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((rank, ws, r, local, t, w))


def test_two_gloo_ranks_reduce_like_bench():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r_, ws, r, local, t, w) in enumerate(out):
        assert (r_, ws, r, local) == (rank, 2, rank, rank)
        assert t == 2.0 and w == 30.0


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    ws, r, local = bench.dist_setup()
    assert (ws, r, local) == (1, 0, 0)
    assert bench.max_over_ranks(1, 3.5) == 3.5 and bench.sum_over_ranks(1, 2.0) == 2.0
