"""The benchmark's multi-process path on CPU: two gloo ranks run bench's
rendezvous, barrier and max-over-ranks timing helpers (the path torchrun
takes with one process per GPU; here without a GPU)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update({"WORLD_SIZE": str(ws), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    got_ws, got_rank, _, pg = bench.dist_setup()
    bench.barrier(pg)
    t = bench.max_over_ranks(pg, 1.5 + rank)  # rank 1 is the slow one
    bench.barrier(pg)
    q.put((got_ws, got_rank, t))
    pg.destroy_process_group()


def test_two_rank_barrier_and_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(2, 0, 2.5), (2, 1, 2.5)]


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 3.25) == 3.25
    bench.barrier(None)
