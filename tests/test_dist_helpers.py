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


def test_clock_record_prefers_the_fast_samples():
    """The line's clocks take NVML's samples inside the timed loop when there
    are any (a loop of a few ms is shorter than nvidia-smi's period), keep
    nvidia-smi's beside them, and report a reason either source saw."""
    sys.path.insert(0, ROOT)
    import bench
    smi = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 1}
    nv = bench.NvmlSampler.__new__(bench.NvmlSampler)
    nv.samples = [(0.5, 1980.0, 0), (1.0, 2070.0, 0x8), (1.5, 2070.0, 0), (3.0, 900.0, 0x40)]
    nv.max_mhz, nv.period = 2070.0, 5e-4
    got = nv.summary((0.4, 2.0))
    assert got["samples"] == 3 and got["sm_mhz"] == 2070.0 and got["sm_mhz_min"] == 1980.0
    assert got["reasons"] == ["hw_slowdown"]
    rec = bench.clock_record(smi, got, {"samples": 3})
    assert rec["source"] == "nvml" and rec["samples"] == 3
    assert rec["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert rec["nvidia_smi"] == smi and rec["heat_and_timed"] == {"samples": 3}
    assert nv.summary((5.0, 6.0)) is None
    assert bench.clock_record(smi, None, {})["source"] == "nvidia-smi"


def test_nvml_sampler_without_a_driver_records_nothing():
    sys.path.insert(0, ROOT)
    import bench
    with bench.NvmlSampler("no-such-gpu") as nv:
        pass
    assert nv.summary((0.0, 1e12)) is None
