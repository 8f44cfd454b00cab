#!/usr/bin/env python3
"""Throughput of the cloth step on the paper-scale workload.

Workload: 800x800 grid cloth (640,000 nodes, 3,832,002 structural/shear/bend
springs), top row pinned, gravity plus a 2 N/kg sinusoidal wind, colliding
with an 81,920-triangle displaced icosphere (radius 0.25 m) -- the stand-in
for the paper's 100K-triangle model; dt = 1/1200 s in 4 substeps.  A "step"
is one cloth_step: 4 fused substep launches (forces, symplectic Euler, grid
broad phase, MT narrow phase, response) over all nodes.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is whole-job node-steps/s with the state
resident in HBM (per-step CUDA events on the library's stream, L2 flushed by
a 256 MiB write before every timed step).  The timed window starts at step
600 of the workload, with the cloth resting on the mesh, so every timed step
runs the narrow phase and the response; `collision` gives the listed nodes,
candidate tests and hit nodes per substep of the window.  `e2e` is the same
metric through the C ABI with pinned host buffers copied in and out every
step (the input is the window's starting state).  `configs` times the other
synthetic workloads over their configured steps next to the FP64 oracle.
Under torchrun every rank steps its own replica of the cloth (no exchange).
`--impl reference` times the FP64 CPU oracle on the host on a bounded row
band of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "node-steps/s at 640K nodes + 100K-tri collision; HBM roofline %; adjoint vs fwd"
UNIT = "node-steps/s"
BYTES_PER_NODE_SUBSTEP = 48  # read p, v (24 B) + write p, v (24 B), float32 SoA
START_STEP = 600    # the timed window starts here (the cloth rests on the mesh)
HEAT_STEPS = 300    # untimed steps just before it, under the clock sampler
LAUNCHES_PER_SUBSTEP = 2  # walk + collision kernel
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "substep_kernel_800x800_l6.txt")
STEP_SRC = os.path.join(ROOT, "paper_2507_11794_gb300", "csrc", "cloth_step.cu")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched, adjoint and atomic A/B legs")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=0, help="steps of the e2e leg (default: --steps, max 1000)")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="run only the adjoint leg and print its result (for profiling the rollout)")
    ap.add_argument("--case", default=None, choices=sorted(CASES),
                    help="run one short fixed workload of a kernel family (for profiler captures) and exit")
    return ap.parse_args()


def workload_config(sc):
    return {"start_step": START_STEP,
        "workload": "800x800 grid cloth (640,000 nodes, 3,832,002 springs), top row pinned, gravity + 2 N/kg "
                    "sinusoidal wind, vs 81,920-triangle displaced icosphere r=0.25 m; dt=1/1200 s, 4 substeps",
        "nodes": sc.n, "springs": 3832002, "triangles": int(sc.ntris), "substeps_per_step": sc.substeps,
        "dt": sc.dt, "l2": "flushed (256 MiB write) before every timed step",
        "timed_window": f"steps {START_STEP}.. of the workload (contact phase), after {START_STEP} untimed steps "
                        "from its initial state",
        "parallelism": "replicas",
    }


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return None


def code_hash(path: str) -> str:
    """sha256 (16 hex digits) of a C/CUDA source with its comments and
    whitespace removed: the same for edits that do not change the code."""
    import re
    src = open(path, encoding="utf-8").read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = re.sub(r"\s+", "", src)
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def profile_traffic():
    """Per-launch DRAM bytes of the substep kernel from the committed ncu
    summary, if it was taken on the current kernel code (comment and
    whitespace changes aside)."""
    try:
        src_hash = code_hash(STEP_SRC)
        vals = {}
        for line in open(PROFILE_SUMMARY):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals.setdefault(k.strip(), v.strip())  # the first block is the benchmarked kernel
        if vals.get("code_sha256_16", "").split()[:1] == [src_hash] and "dram_bytes_per_launch" in vals:
            return float(vals["dram_bytes_per_launch"])
    except (OSError, ValueError):
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled while the timed loop runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.rows = []
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "20"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi takes a while to start: wait for its first sample so the
            # timed region is covered
            t_end = time.perf_counter() + 5.0
            while not self.rows and time.perf_counter() < t_end and self.proc.poll() is None:
                time.sleep(0.01)
        except OSError:
            self.proc = None
        self.window = None
        return self

    def mark(self, t0: float, t1: float):
        """The timed region, in time.perf_counter() seconds."""
        self.window = (t0, t1)

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")] + [time.perf_counter()])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, window=None):
        """Median SM clock, max clock and active slowdown reasons over the
        samples taken inside a window (default: the marked timed region),
        plus the sample either side of it, which brackets a window shorter
        than the sampling period."""
        rows = [r for r in self.rows if len(r) >= 10]
        window = window or self.window
        if window is not None and rows:
            t0, t1 = window
            inside = [i for i, r in enumerate(rows) if t0 <= r[-1] <= t1]
            before = [i for i, r in enumerate(rows) if r[-1] < t0][-1:]
            after = [i for i, r in enumerate(rows) if r[-1] > t1][:1]
            rows = [rows[i] for i in before + inside + after]
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                mhz.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for nm, val in zip(names, r[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        mhz.sort()
        return {"sm_mhz": mhz[len(mhz) // 2] if mhz else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


class NvmlSampler:
    """SM clock and clock-event reasons read through NVML (the driver's
    libnvidia-ml, read-only queries) by a thread polling every `period_s`
    while the timed loop runs: nvidia-smi's own loop samples about every
    20 ms, longer than a timed loop of a few milliseconds."""

    # clock-event reason bits of nvmlDeviceGetCurrentClocksEventReasons
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, uuid: str | None, period_s: float = 5e-4):
        self.samples = []  # (perf_counter, sm MHz, reason bits)
        self.period = period_s
        self.dev = None
        self.max_mhz = None
        self.stop = threading.Event()
        try:
            import ctypes as C
            self.C = C
            self.lib = C.CDLL("libnvidia-ml.so.1")
            if self.lib.nvmlInit_v2() != 0:
                return
            n = C.c_uint(0)
            self.lib.nvmlDeviceGetCount_v2(C.byref(n))
            want = (uuid or "").lower().replace("gpu-", "")
            for i in range(n.value):
                h = C.c_void_p()
                if self.lib.nvmlDeviceGetHandleByIndex_v2(i, C.byref(h)) != 0:
                    continue
                buf = C.create_string_buffer(96)
                self.lib.nvmlDeviceGetUUID(h, buf, 96)
                if not want or buf.value.decode().lower().replace("gpu-", "") == want:
                    self.dev = h
                    break
            if self.dev is not None:
                m = C.c_uint(0)
                if self.lib.nvmlDeviceGetMaxClockInfo(self.dev, 1, C.byref(m)) == 0:
                    self.max_mhz = float(m.value)
                self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                    self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        except (OSError, AttributeError):
            self.dev = None

    def _poll(self):
        C = self.C
        mhz, bits = C.c_uint(0), C.c_ulonglong(0)
        while not self.stop.is_set():
            ok = self.lib.nvmlDeviceGetClockInfo(self.dev, 1, C.byref(mhz)) == 0
            ok = ok and self.reasons_fn(self.dev, C.byref(bits)) == 0
            if ok:
                self.samples.append((time.perf_counter(), float(mhz.value), int(bits.value)))
            time.sleep(self.period)

    def __enter__(self):
        if self.dev is not None:
            self.t = threading.Thread(target=self._poll, daemon=True)
            self.t.start()
        return self

    def __exit__(self, *exc):
        if self.dev is not None:
            self.stop.set()
            self.t.join(timeout=5)

    def summary(self, window):
        t0, t1 = window
        inside = [s for s in self.samples if t0 <= s[0] <= t1]
        if not inside:
            return None
        mhz = sorted(s[1] for s in inside)
        reasons = sorted(nm for nm, b in self.BITS.items() if any(s[2] & b for s in inside))
        return {"sm_mhz": mhz[len(mhz) // 2], "sm_mhz_min": mhz[0], "sm_max_mhz": self.max_mhz, "reasons": reasons,
                "samples": len(mhz), "period_ms": self.period * 1e3}


def clock_record(smi: dict, nvml: dict | None, heat: dict) -> dict:
    """The line's clocks: NVML's samples inside the timed loop where there
    are any (median SM clock, union of the reasons seen), else nvidia-smi's;
    nvidia-smi's samples of the timed loop (with the one either side) and of
    the heat-up plus timed steps are kept beside them."""
    out = dict(nvml) if nvml else dict(smi)
    out["source"] = "nvml" if nvml else "nvidia-smi"
    if nvml:
        out["reasons"] = sorted(set(nvml["reasons"]) | set(smi.get("reasons") or []))
    out["nvidia_smi"] = smi
    out["heat_and_timed"] = heat
    return out


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return ws, rank, local, pg


def barrier(pg):
    import torch
    if pg is not None:
        if torch.cuda.is_available():
            pg.barrier(device_ids=[torch.cuda.current_device()])
        else:
            pg.barrier()


def max_over_ranks(pg, x: float) -> float:
    if pg is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def host_cpu():
    """CPU model and logical core count of this host."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":", 1)[0].strip().lower()
                if k in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"cpu_model": model or platform.machine(), "nproc": os.cpu_count()}


def oracle_rate(sc, steps: int, rows: int | None = None):
    """Node-steps/s of the FP64 oracle (1 thread) on the first `rows` rows of
    a scene (all rows by default) for `steps` steps from its initial state,
    with the scene's own mesh.  Returns (rate, seconds, nodes)."""
    import dataclasses

    import numpy as np

    import oracle
    rows = sc.ny if rows is None else min(rows, sc.ny)
    nx = sc.nx
    sub = dataclasses.replace(sc, ny=rows, init_pos=sc.init_pos[:rows * nx], init_vel=sc.init_vel[:rows * nx],
                              pinned=sc.pinned[:rows * nx])
    cl = oracle.Cloth(sub)
    grid = oracle.Grid(sub.mesh_verts, sub.mesh_tris) if sub.mesh_tris is not None else None
    x, v = sub.init_pos, sub.init_vel
    t0 = time.perf_counter()
    x, v = oracle.step(cl, x, v, 0, steps * sub.substeps, grid)
    dt = time.perf_counter() - t0
    assert np.all(np.isfinite(x))
    return rows * nx * steps / dt, dt, rows * nx


def cpu_oracle_sample(sc, rows: int, steps: int):
    """Time the FP64 oracle on the first `rows` rows of the cloth for `steps`
    steps (1 thread).  Returns (node-steps/s, seconds, nodes)."""
    import dataclasses

    import numpy as np

    import oracle
    nx = sc.nx
    sub = dataclasses.replace(sc, ny=rows, init_pos=sc.init_pos[:rows * nx], init_vel=sc.init_vel[:rows * nx],
                              pinned=sc.pinned[:rows * nx])
    cl = oracle.Cloth(sub)
    grid = oracle.Grid(sub.mesh_verts, sub.mesh_tris)
    x, v = sub.init_pos, sub.init_vel
    t0 = time.perf_counter()
    for s in range(steps):
        x, v = oracle.step(cl, x, v, s * sub.substeps, sub.substeps, grid)
    dt = time.perf_counter() - t0
    assert np.all(np.isfinite(x))
    return rows * nx * steps / dt, dt, rows * nx


def cpu_oracle_band(sc, x, v, row0: int, rows: int, steps: int, k0: int):
    """Time the FP64 oracle (1 thread) on rows [row0, row0 + rows) of the
    cloth, started from the given float32 state at global substep k0, with
    the full mesh, for `steps` steps.  Returns (node-steps/s, seconds, nodes)."""
    import dataclasses

    import numpy as np

    import oracle
    nx = sc.nx
    sl = slice(row0 * nx, (row0 + rows) * nx)
    sub = dataclasses.replace(sc, ny=rows, init_pos=np.ascontiguousarray(x[sl]), init_vel=np.ascontiguousarray(v[sl]),
                              pinned=np.ascontiguousarray(sc.pinned[sl]),
                              origin=tuple(float(sc.origin[a] + row0 * sc.dv[a]) for a in range(3)))
    cl = oracle.Cloth(sub)
    grid = oracle.Grid(sub.mesh_verts, sub.mesh_tris)
    t0 = time.perf_counter()
    xo, _ = oracle.step(cl, sub.init_pos, sub.init_vel, k0, steps * sub.substeps, grid)
    dt = time.perf_counter() - t0
    assert np.all(np.isfinite(xo))
    return rows * nx * steps / dt, dt, rows * nx


def run_config_legs(stream, flush, peak):
    """The other synthetic workloads, each over its configured steps from its
    initial state (per-step CUDA events, L2 flushed before every step):
    node-steps/s, the whole-step HBM fraction (48 B per node-substep over the
    step time) and the FP64 oracle's rate on a bounded sample (1 thread)."""
    import numpy as np
    import torch

    import cloth_scenes as cs
    import paper_2507_11794_gb300 as P
    legs = {}
    specs = [("config1_32x32_L2", cs.config1(), None, 200),
             ("config2_256x256_L6", cs.config2(), None, 30),
             ("config3i_800x800_none", cs.config3("none"), 400, 30),
             ("config3ii_800x800_L5", cs.config3("l5"), 400, 30)]
    for name, sc, rows, osteps in specs:
        cl = P.Cloth(sc, stream=int(stream.cuda_stream))
        cl.step(2)
        cl.set_state(sc.init_pos, sc.init_vel)
        cl.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(sc.steps)]
        for i in range(sc.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            cl.step(1)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / sc.steps
        listed, tested, hits = cl.collision_stats()
        pos, _ = cl.read()
        assert np.all(np.isfinite(pos))
        cl.close()
        val = sc.n / (ms / 1e3)
        achieved = BYTES_PER_NODE_SUBSTEP * sc.n * sc.substeps / (ms * 1e-3) / 1e9
        orate, odt, onodes = oracle_rate(sc, osteps, rows)
        nsub = sc.steps * sc.substeps
        legs[name] = {"nodes": sc.n, "triangles": sc.ntris, "steps": sc.steps, "substeps_per_step": sc.substeps,
                      "ms_per_step": ms, "node_steps_per_s": val,
                      "node_substeps_per_s": val * sc.substeps,
                      "hbm_frac_whole_step": achieved / peak, "achieved_gbs_whole_step": achieved,
                      "mean_listed_per_substep": listed / (nsub + 2 * sc.substeps),
                      "mean_tested_per_substep": tested / (nsub + 2 * sc.substeps),
                      "oracle_node_steps_per_s": orate,
                      "oracle_sample": f"{'all' if rows is None else f'first {rows}'} rows ({onodes} nodes), "
                                       f"{osteps} steps from the initial state, FP64, 1 thread, {odt:.1f} s",
                      "gpu_over_oracle": val / orate}
    return legs


def run_reference(args):
    ws, rank, _, pg = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0, None
    if rank != 0:
        return 0
    import cloth_scenes as cs
    import oracle
    oracle.build()
    sc = cs.config3("l6")
    # calibrate: one step of a 16-row band, then size the band so the whole
    # --steps + --warmup run stays within about two minutes
    _, t16, _ = cpu_oracle_sample(sc, 16, 1)
    budget = 120.0 / max(1, args.steps + args.warmup)
    rows = int(max(4, min(sc.ny, 16 * budget / max(t16, 1e-6))))
    cpu_oracle_sample(sc, rows, max(0, min(args.warmup, 3)))
    val, dt, nodes = cpu_oracle_sample(sc, rows, args.steps)
    sample = (f"first {rows} rows ({nodes} nodes) of the 800x800 cloth with the full 81,920-triangle mesh, "
              f"{args.steps} steps x 4 substeps from the initial state, FP64 oracle, 1 thread")
    out = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(1, args.steps), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(sc), "impl": "reference",
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def run_batch(args, stream):
    """The batched workload: 256 cloths of uneven size (9.3M nodes), each with
    its own displaced icosphere (1,280-81,920 triangles), 10 substeps per
    step; one persistent walk + one collision launch per substep (autotuned),
    against the same cloths stepped by one cloth_step each."""
    import numpy as np
    import torch

    import cloth_scenes as cs
    import paper_2507_11794_gb300 as P
    scenes = cs.config5()
    nodes = sum(s.n for s in scenes)
    sub = scenes[0].substeps
    b = P.ClothBatch(scenes, stream=int(stream.cuda_stream))
    tuning = b.tune(10)
    b.step(2)
    b.sync()
    stats0 = b.collision_stats()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    b.step(args.batch_steps)
    ev[1].record(stream)
    torch.cuda.synchronize()
    t_batch = ev[0].elapsed_time(ev[1]) / 1e3
    stats1 = b.collision_stats()
    nsub = args.batch_steps * sub
    coll = {"listed_per_substep": (stats1[0] - stats0[0]) / nsub,
            "tested_per_substep": (stats1[1] - stats0[1]) / nsub,
            "hit_nodes_per_substep": (stats1[2] - stats0[2]) / nsub}
    for i in range(len(scenes)):
        p, _ = b.read(i)
        assert np.all(np.isfinite(p))
    b.close()
    singles = [P.Cloth(s, stream=int(stream.cuda_stream)) for s in scenes]
    for c in singles:
        c.step(1)
    torch.cuda.synchronize()
    ks = max(2, args.batch_steps // 4)
    ev[0].record(stream)
    for _ in range(ks):
        for c in singles:
            c.step(1)
    ev[1].record(stream)
    torch.cuda.synchronize()
    t_single = ev[0].elapsed_time(ev[1]) / 1e3
    for c in singles:
        c.close()
    batch_val = nodes * args.batch_steps / t_batch
    single_val = nodes * ks / t_single
    us_sub = 1e6 * t_batch / (args.batch_steps * sub)
    achieved = BYTES_PER_NODE_SUBSTEP * nodes / (us_sub * 1e-6) / 1e9
    peaks = measured_peaks()
    peak = float(peaks["hbm_gbs"]) if peaks and "hbm_gbs" in peaks else 6800.0
    return {"workload": f"256 cloths, sides 16-512 log-uniform (seed 1), {nodes} nodes, each over its own "
                        f"displaced icosphere (1,280-81,920 triangles); dt=1/1200 s, {sub} substeps per step",
            "metric": "node-steps/s", "value": batch_val, "steps": args.batch_steps,
            "ms_per_step": 1e3 * t_batch / args.batch_steps,
            "per_cloth_launch_value": single_val, "per_cloth_launch_steps": ks,
            "speedup_vs_per_cloth_launches": batch_val / single_val,
            "tuning": {"rows_per_warp": tuning.rows_per_warp, "walk_ctas_per_sm": tuning.walk_ctas_per_sm,
                       "candidates": tuning.candidates},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "scope": "walk + collision launches of one substep",
                         "algorithmic_bytes_per_substep": BYTES_PER_NODE_SUBSTEP * nodes},
            "collision": coll, "l2": "state (446 MB per substep) larger than L2"}


def run_adjoint(stream):
    """Differentiation workload: 128x128 cloth over a 5,120-triangle icosphere,
    256-step rollout with checkpoints every 16 steps; times the forward pass
    and the reverse pass (gradients w.r.t. per-spring ks, kd and v0)."""
    import torch

    import cloth_scenes as cs
    import paper_2507_11794_gb300 as P
    from paper_2507_11794_gb300.rollout import Rollout
    sc = cs.config4()
    cl = P.Cloth(sc, stream=int(stream.cuda_stream))
    ro = Rollout(cl, sc.steps, 16)
    ks = torch.tensor(sc.ks_spring, device="cuda", requires_grad=True)
    kd = torch.tensor(sc.kd_spring, device="cuda", requires_grad=True)
    v0 = torch.tensor(sc.init_vel, device="cuda", requires_grad=True)
    tgt = torch.tensor(sc.init_pos, device="cuda")
    fw, bw = [], []
    for it in range(3):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        pos, _ = ro(ks, kd, v0)
        ev[1].record(stream)
        loss = ((pos - tgt) ** 2).sum(1).mean()
        loss.backward()
        ev[2].record(stream)
        torch.cuda.synchronize()
        if it > 0:
            fw.append(ev[0].elapsed_time(ev[1]))
            bw.append(ev[1].elapsed_time(ev[2]))
        ks.grad = kd.grad = v0.grad = None
    ro.close()
    cl.close()
    f, b = min(fw), min(bw)
    return {"workload": "128x128 cloth (16,384 nodes, 97,026 springs) over a 5,120-triangle icosphere, 256-step "
                        "rollout, checkpoints every 16 steps, grads w.r.t. per-spring ks, kd and v0",
            "forward_ms": f, "backward_ms": b, "backward_over_forward": b / f,
            "forward_node_steps_per_s": sc.n * sc.steps / (f / 1e3)}


def run_atomic_ab(stream, flush, steps: int = 100):
    """The paper's force pass (Algorithm 1: one thread per spring, FP32
    atomic adds, then a per-node integration kernel) against the fused column
    walk, on the benchmark workload: the first `steps` steps from the initial
    state, L2 flushed before each, per-step CUDA events; then per-kernel
    times over 20 more steps."""
    import torch

    import cloth_scenes as cs
    import paper_2507_11794_gb300 as P
    sc = cs.config3("l6")
    out = {"workload": f"the benchmark workload, first {steps} steps from the initial state, L2 flushed per step"}
    for name, flags in (("fused_walk", 0), ("atomic_springs", P.capi.CLOTH_FLAG_ATOMIC_SPRINGS)):
        cl = P.Cloth(sc, stream=int(stream.cuda_stream), flags=flags)
        for _ in range(3):
            cl.step(1)
        cl.set_state(sc.init_pos, sc.init_vel)
        cl.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            cl.step(1)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        w = c = 0.0
        for i in range(20):
            flush.fill_(float(i))
            wi, ci = cl.profile_substeps(sc.substeps)
            w += wi / 20
            c += ci / 20
        cl.close()
        out[name] = {"node_steps_per_s": sc.n * steps / (ms / 1e3), "ms_per_step": ms / steps,
                     "force_integrate_us_per_substep": w, "collide_us_per_substep": c}
    out["fused_over_atomic"] = out["fused_walk"]["node_steps_per_s"] / out["atomic_springs"]["node_steps_per_s"]
    return out


def run_edge_ab(stream, flush, warm: int = 150, steps: int = 100):
    """The paper's own narrow phase (cloth-triangle edges against the surface,
    CLOTH_FLAG_EDGE_COLLISION) against the default node-path narrow phase on
    the 256x256 cloth over the 81,920-triangle mesh: steps `warm`..`warm+steps`
    (the cloth lands on the mesh), L2 flushed before each step."""
    import torch

    import cloth_scenes as cs
    import paper_2507_11794_gb300 as P
    sc = cs.config2()
    out = {"workload": f"256x256 cloth (65,536 nodes) over the 81,920-triangle displaced icosphere, steps "
                       f"{warm}-{warm + steps} (contact), dt=1/1200 s, 4 substeps, L2 flushed per step"}
    for name, flags in (("node_paths", 0), ("edges", P.capi.CLOTH_FLAG_EDGE_COLLISION)):
        cl = P.Cloth(sc, stream=int(stream.cuda_stream), flags=flags)
        cl.step(warm)
        cl.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            cl.step(1)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        w = c = 0.0
        for i in range(10):
            flush.fill_(float(i))
            wi, ci = cl.profile_substeps(sc.substeps)
            w += wi / 10
            c += ci / 10
        cl.close()
        out[name] = {"ms_per_step": ms, "node_steps_per_s": sc.n / (ms / 1e3), "walk_us_per_substep": w,
                     "collision_us_per_substep": c}
    return out


def run_pulling(stream, flush, warm: int = 150, steps: int = 150):
    """The paper's second experiment: a 256x256 cloth (65,536 nodes) pulled
    by its pinned leading row at 0.5 m/s across the 81,920-triangle model;
    steps warm..warm+steps (the cloth slides over the model), L2 flushed
    before each step."""
    import torch

    import cloth_scenes as cs
    import paper_2507_11794_gb300 as P
    sc = cs.pulling_scene(256, "l6")
    cl = P.Cloth(sc, stream=int(stream.cuda_stream))
    cl.step(warm)
    cl.sync()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        cl.step(1)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    cl.close()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    return {"workload": f"256x256 cloth (65,536 nodes) pulled at 0.5 m/s across the 81,920-triangle model, steps "
                        f"{warm}-{warm + steps}, dt=1/1200 s in 4 substeps, L2 flushed per step",
            "ms_per_step": ms, "node_steps_per_s": sc.n / (ms / 1e3), "steps_per_s": 1e3 / ms}


def run_ours(args):
    import numpy as np
    import torch

    import cloth_scenes as cs
    import paper_2507_11794_gb300 as P
    from paper_2507_11794_gb300 import build as B

    ws, rank, local, pg = dist_setup()
    if rank == 0 or pg is None:
        B.build()
    barrier(pg)
    sc = cs.config3("l6")
    N, SUB = sc.n, sc.substeps
    stream = torch.cuda.current_stream()
    cl = P.Cloth(sc, stream=int(stream.cuda_stream))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        flush.fill_(1.0)
        cl.step(1)
    cl.sync()
    # the timed window starts in the contact phase: from the workload's
    # initial state, START_STEP steps run untimed, the last HEAT of them with
    # the same L2 flushes as the timed steps (the clock sampler covers them)
    cl.set_state(sc.init_pos, sc.init_vel)
    heat = min(HEAT_STEPS, START_STEP)
    cl.step(START_STEP - heat)
    cl.sync()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    try:
        uuid = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    except (AttributeError, RuntimeError):
        uuid = None
    with ClockSampler(torch.cuda.current_device()) as clocks, NvmlSampler(uuid) as nv:
        h0 = time.perf_counter()
        for i in range(heat):
            flush.fill_(float(i))
            cl.step(1)
        stats0 = cl.collision_stats()  # synchronises
        x_start, v_start = cl.read()
        barrier(pg)
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(float(i))
            starts[i].record(stream)
            cl.step(1)
            ends[i].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        clocks.mark(wall0, wall0 + wall)
    barrier(pg)
    stats1 = cl.collision_stats()
    nsub_timed = args.steps * SUB
    coll = {"listed_per_substep": (stats1[0] - stats0[0]) / nsub_timed,
            "tested_per_substep": (stats1[1] - stats0[1]) / nsub_timed,
            "hit_nodes_per_substep": (stats1[2] - stats0[2]) / nsub_timed}
    dev_ms = sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends))
    pos, vel = cl.read()
    assert np.all(np.isfinite(pos)) and np.all(np.isfinite(vel))
    t = max_over_ranks(pg, dev_ms / 1e3)
    value = ws * N * args.steps / t
    launches = LAUNCHES_PER_SUBSTEP * SUB * args.steps

    # kernel split: the same steps (L2 flushed before each), every kernel
    # launch bracketed by CUDA events on the library's stream; the events
    # stop each launch from overlapping the previous one's tail, so these
    # durations only give the walk's share of the substep, which is applied
    # to the timed substep
    prof_steps = min(args.steps, 200)
    walk_ev = coll_ev = 0.0
    for i in range(prof_steps):
        flush.fill_(float(i))
        w, c = cl.profile_substeps(SUB)
        walk_ev += w / prof_steps
        coll_ev += c / prof_steps

    # end to end through the C ABI: pinned host state in (the contact-phase
    # state the timed window started from), step, state out
    ke = args.e2e_steps or min(args.steps, 1000)
    hp = torch.empty((N, 3), dtype=torch.float32, pin_memory=True).numpy()
    hv = torch.empty((N, 3), dtype=torch.float32, pin_memory=True).numpy()
    op = torch.empty((N, 3), dtype=torch.float32, pin_memory=True).numpy()
    ov = torch.empty((N, 3), dtype=torch.float32, pin_memory=True).numpy()
    hp[:] = x_start
    hv[:] = v_start
    barrier(pg)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(ke):
        cl.set_state(hp, hv)
        cl.step(1)
        cl.read(out_pos=op, out_vel=ov)
    e2e_t = max_over_ranks(pg, time.perf_counter() - e0)
    e2e_val = ws * N * ke / e2e_t

    # per-vertex normals of the final state (the pre-render update), L2 flushed before each call
    nrm = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    nev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(50)]
    for i, (a, b) in enumerate(nev):
        flush.fill_(float(i))
        a.record(stream)
        cl.normals(nrm)
        b.record(stream)
    torch.cuda.synchronize()
    nrm_us = 1e3 * min(a.elapsed_time(b) for a, b in nev)
    normals = {"kernel": "normals_kernel", "us": nrm_us, "algorithmic_bytes": 24 * N,
               "achieved_gbs": 24 * N / (nrm_us * 1e-6) / 1e9,
               "timing": "CUDA events around each of 50 calls after a 256 MiB L2 flush; best call"}
    cl.close()
    batch = None if args.no_batch else run_batch(args, stream)
    adjoint = None if args.no_batch else run_adjoint(stream)
    atomic_ab = None if args.no_batch else run_atomic_ab(stream, flush)
    edge_ab = None if args.no_batch else run_edge_ab(stream, flush)
    pulling = None if args.no_batch else run_pulling(stream, flush)
    if rank != 0:
        if pg is not None:
            pg.destroy_process_group()
        return 0

    peaks = measured_peaks()
    peak = float(peaks["hbm_gbs"]) if peaks and "hbm_gbs" in peaks else 6800.0
    normals["frac"] = normals["achieved_gbs"] / peak
    peak_src = "measured" if peaks and "hbm_gbs" in peaks else "fallback"
    us_sub = 1e3 * (t / args.steps) * 1e3 / SUB  # timed substep, us
    share = walk_ev / (walk_ev + coll_ev) if walk_ev + coll_ev > 0 else 1.0
    walk_us = us_sub * share
    achieved = BYTES_PER_NODE_SUBSTEP * N / (walk_us * 1e-6) / 1e9
    step_achieved = BYTES_PER_NODE_SUBSTEP * N / (us_sub * 1e-6) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": profile_traffic(), "peak_source": peak_src,
                "kernel": "substep_kernel<MESH=true> (walk: springs + integration)",
                "algorithmic_bytes_per_launch": BYTES_PER_NODE_SUBSTEP * N,
                "avg_launch_us": walk_us,
                "timing": "timed substep (ms_per_step / substeps) x the walk's share of the substep's kernel time; "
                          "the share is from event-bracketed launches over the next steps",
                "walk_share": share, "event_bracketed_walk_us": walk_ev, "event_bracketed_collide_us": coll_ev,
                "whole_substep": {"us": us_sub, "achieved": step_achieved, "frac": step_achieved / peak}}
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        row0, rows, csteps = 280, 400, 10
        val, dt, nodes = cpu_oracle_band(sc, x_start, v_start, row0, rows, csteps, START_STEP * SUB)
        cpu = {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", **host_cpu(),
               "sample": f"rows {row0}-{row0 + rows - 1} ({nodes} nodes) of the cloth's float32 state at step "
                         f"{START_STEP} (the timed window's start, in contact with the mesh), {csteps} steps x 4 "
                         f"substeps with the full mesh ({dt:.1f} s, FP64, 1 thread)"}
    legs = None if args.no_batch else run_config_legs(stream, flush, peak)
    heat_clocks = clocks.summary((h0, wall0 + wall))
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": workload_config(sc),
           "roofline": roofline, "cpu_baseline": cpu,
           "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 2 * 12 * N,
                   "d2h_bytes_per_step": 2 * 12 * N, "steps": ke},
           "gpu_launches": launches,
           "clocks": clock_record(clocks.summary(), nv.summary((wall0, wall0 + wall)), heat_clocks),
           "collision": coll, "batch": batch, "adjoint": adjoint, "atomic_springs_ab": atomic_ab,
           "edge_narrow_phase_ab": edge_ab, "pulling_scene": pulling, "configs": legs,
           "normals": normals,
           "wall_s_timed_loop": wall}
    print(json.dumps(out), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


def run_case(name: str):
    """Short fixed workloads, one per kernel family, for profiler captures
    (ncu -k <kernel> -s <skip> -c <count> python bench.py --case NAME); each
    prints one line with the launches it made."""
    import torch

    import cloth_scenes as cs
    import paper_2507_11794_gb300 as P
    from paper_2507_11794_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)
    if name in ("walk", "collide"):
        # the benchmark workload in contact: 600 steps, then 2 more
        sc = cs.config3("l6")
        cl = P.Cloth(sc)
        cl.step(START_STEP + 2)
        cl.sync()
        info = f"{(START_STEP + 2) * sc.substeps} launches of each of substep_kernel and collide_kernel"
    elif name == "walk_none":
        sc = cs.config3("none")
        cl = P.Cloth(sc)
        cl.step(3)
        cl.sync()
        info = f"{3 * sc.substeps} launches of substep_kernel"
    elif name == "batch":
        b = P.ClothBatch(cs.config5())
        b.set_tuning(24, b.tuning().walk_ctas_per_sm)  # the autotuner's usual pick, fixed
        b.step(2)
        b.sync()
        info = ("batch without autotuning (24 rows per warp, the default walk CTAs per SM): 2 steps x 10 "
                "substeps of batch_substep_kernel + batch_collide_kernel")
    elif name == "grid":
        sc = cs.config3("l6")
        cl = P.Cloth(sc, mesh=False)
        cl.set_mesh(sc.mesh_verts, sc.mesh_tris)
        cl.sync()
        info = "one grid build over the 81,920-triangle mesh"
    elif name == "normals":
        sc = cs.config3("none")
        cl = P.Cloth(sc)
        cl.step(3)
        out = torch.empty((sc.n, 3), device="cuda")
        for _ in range(3):
            cl.normals(out)
        torch.cuda.synchronize()
        info = "12 substeps, then 3 launches of normals_kernel"
    elif name == "atomic":
        sc = cs.config3("l6")
        cl = P.Cloth(sc, flags=P.capi.CLOTH_FLAG_ATOMIC_SPRINGS)
        cl.step(3)
        cl.sync()
        info = "3 steps of the atomic spring path (spring_atomic_kernel, node_integrate_kernel, collide_kernel)"
    elif name == "adjoint":
        from paper_2507_11794_gb300.rollout import Rollout
        sc = cs.config4()
        cl = P.Cloth(sc)
        ro = Rollout(cl, 32, 16)
        ks = torch.tensor(sc.ks_spring, device="cuda", requires_grad=True)
        kd = torch.tensor(sc.kd_spring, device="cuda", requires_grad=True)
        v0 = torch.tensor(sc.init_vel, device="cuda", requires_grad=True)
        pos, _ = ro(ks, kd, v0)
        (pos ** 2).sum().backward()
        torch.cuda.synchronize()
        ro.close()
        info = "a 32-step rollout of the differentiation workload, forward and backward (adj_kernel)"
    else:  # edges
        sc = cs.config2()
        cl = P.Cloth(sc, flags=P.capi.CLOTH_FLAG_EDGE_COLLISION)
        cl.step(240)
        cl.sync()
        info = ("240 steps (960 substeps; contact from about step 160) of the 256x256 cloth over the "
                "81,920-triangle mesh with the edge narrow phase")
    print(json.dumps({"case": name, "launches": info}), flush=True)
    return 0


CASES = ("walk", "collide", "walk_none", "batch", "grid", "normals", "atomic", "adjoint", "edges")


def main():
    args = parse()
    if args.case:
        return run_case(args.case)
    if args.impl == "reference":
        return run_reference(args)
    if args.adjoint_only:
        import torch
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            print(json.dumps({"adjoint": run_adjoint(stream)}), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
