"""Benchmark: light samples per second of one learning pass (sample + shade +
shadow + learn + split-collapse) on the frame-scale static scene
(1920 x 1080 G-buffer, 64K emissive triangles in 64 patches, 64 occluder
boxes, 2^20-entry hash grid, cut size 32, 1 sample per point).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line. A step is one full pass over the frame. Inputs are
resident in device memory; L2 is flushed (512 MB write) between timed steps,
outside the timed region; every step is timed with CUDA events on the
library's stream. `e2e` repeats the measurement through the host-buffer C
entry point (G-buffer uploaded and rgb read back inside the timed region).
With --impl reference the CPU oracle is timed on a bounded slice of the same
workload (there is no other implementation of the method to run).
Under torchrun each rank renders its own replica (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("light samples/sec (sample+shade+shadow+learn) at 1 GB300; MSE at equal spp; "
          "p99 frame ms")
UNIT = "light samples/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
SM_COUNT = 152
# DRAM bytes (read + write) of one k_sample launch on this workload, from one ncu capture of it
# (76.30 MB read + 20.90 MB written; kernel as of commit e94a3a1); None whenever the sampling
# kernel has changed since that capture
K_SAMPLE_DRAM_BYTES = 97.19e6
FP32_LANES_PER_SM = 128


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except OSError:
        return dict(PEAKS_FALLBACK, sm_max_mhz=2070.0), "fallback"


def workload_config(scene, tree="lbvh", mode="descent"):
    g = scene.grid
    return {"workload": "frame-scale static walled-cells scene, 1920x1080 G-buffer on 16 planes, "
                        "64K emissive triangles in 64 patches, 64 occluder boxes, one learning pass "
                        "(sample+shade+shadow, Eq.1, Eq.2, split-collapse) per step",
            "points": scene.n_points, "lights": scene.n_lights, "boxes": int(scene.boxes.shape[0]),
            "spp": scene.spp, "cut_size": g.cut_size, "table_size": g.table_size,
            "cell_size": g.cell_size, "normal_bins": g.normal_bins, "jitter": g.jitter,
            "table_precision": "fp32", "in_cluster": mode, "split_iterations": g.split_iterations,
            "light_tree": {"lbvh": "radix tree of Morton codes", "saoh": "Morton order, SAOH split positions",
                       "median": "Morton order, median split positions"}[tree],
            "l2": "flushed between timed steps (512 MB write, untimed)"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def ops_per_sample(n_boxes, n_lights, m):
    """Algorithmic binary32 operations of one light sample (the count used
    for the ALU roofline of the sampling kernel): 18 per slab-tested box
    (6 fma, 12 min/max/compare), 90 per descent level (two node importances
    of ~45 operations), descent depth log2(N / m), and 250 for hashing, the
    cdf search, Philox, the triangle point and shading."""
    levels = max(0.0, math.log2(max(1.0, n_lights / max(1, m))))
    return 18 * n_boxes + 90 * levels + 250


def bytes_per_sample():
    """Algorithmic HBM bytes of one sample in the sampling kernel: G-buffer
    28 B read (position, normal, albedo), rgb 12 B and record 8 B written."""
    return 28 + 12 + 8


def learn_step_bytes(n_records, touched_cells, cut_size, precision="fp32"):
    """Algorithmic HBM bytes of one learning step (Eq. 1, split-collapse,
    Eq. 2): every 8-byte record (key, reward) read once, and per touched cell
    its rows: node ids read and written (8 B per leaf), Q read, Q and C
    written (3 table entries per leaf) -- 20 B per leaf with binary32 tables,
    14 B with 16-bit Q and C."""
    per_leaf = 8 + 3 * (4 if precision == "fp32" else 2)
    return 8 * n_records + per_leaf * cut_size * touched_cells


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_replica(rank, workers, seed, steps, chunk, seconds, barrier, results):
    """One oracle process: the frame workload's points [rank/workers,
    (rank+1)/workers) with its own tree and grid. `seconds` > 0: learning
    passes over consecutive chunks for that long; else `steps` steps, each on
    this process's share of a `chunk`-point slice, started together."""
    from oracle import oracle as O
    from paper_1911_10217_gb300 import scenes
    scene = scenes.frame_scene(seed=seed)
    tree = O.Tree(scene.tris, scene.emission)
    grid = O.Grid.for_scene(tree, scene)
    A = O.scene_arrays(scene)
    P = scene.n_points
    if seconds > 0:
        lo, hi = rank * P // workers, (rank + 1) * P // workers
        start, frame, done = lo, 0, 0
        barrier.wait()
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < seconds:
            cnt = min(chunk, hi - start)
            out = grid.sample_frame(A, scene.seed, frame, scene.spp, first=start, count=cnt)
            grid.learn(out["slot"], out["s"], out["reward"])
            done += cnt * scene.spp
            start += cnt
            if start >= hi:
                start, frame = lo, frame + 1
        results.put((rank, done, time.perf_counter() - t0, []))
        return
    times = []
    chunk = min(chunk, P)
    for i in range(steps):
        first = (i * chunk) % (P - chunk) if chunk < P else 0
        first += rank * chunk // workers
        cnt = (rank + 1) * chunk // workers - rank * chunk // workers
        barrier.wait()
        t0 = time.perf_counter()
        out = grid.sample_frame(A, scene.seed, i, scene.spp, first=first, count=cnt)
        touched = grid.learn(out["slot"], out["s"], out["reward"])
        grid.split_collapse(touched)
        times.append(time.perf_counter() - t0)
    results.put((rank, cnt * steps * scene.spp, sum(times), times))


def _run_replicas(workers, seed, steps=0, chunk=65536, seconds=0.0):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier, results = ctx.Barrier(workers), ctx.Queue()
    procs = [ctx.Process(target=_oracle_replica, args=(r, workers, seed, steps, chunk, seconds, barrier, results))
             for r in range(workers)]
    for p in procs:
        p.start()
    out = [results.get() for _ in procs]
    for p in procs:
        p.join()
    return sorted(out)


def cpu_baseline(scene, single_seconds=6.0, cpu_seconds=24.0, chunk=65536):
    """The oracle on the host cores: one process per core, each on its own
    share of the frame's points with its own grid, learning passes (sample +
    Eq. 1 + Eq. 2) for cpu_seconds / cores seconds (about cpu_seconds of CPU
    work in all); plus one process alone for single_seconds."""
    cores = _host_cores()
    one = _run_replicas(1, scene.seed, chunk=chunk, seconds=single_seconds)[0]
    many = _run_replicas(cores, scene.seed, chunk=chunk // 4, seconds=max(1.0, cpu_seconds / cores))
    done = sum(r[1] for r in many)
    wall = max(r[2] for r in many)
    return {"value": done / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} samples: {cores} oracle processes (one per host core), each learning passes "
                      f"(sample+Eq.1+Eq.2) over consecutive {chunk // 4}-point slices of its own 1/{cores} of "
                      f"the frame-scale workload with its own grid, {wall:.1f} s",
            "single_core": {"value": one[1] / one[2], "cores": 1,
                            "sample": f"{one[1]} samples, one process, {one[2]:.1f} s"}}


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (a job takes as long as its slowest rank);
    x itself without a process group."""
    if not dist:
        return x
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, ms_per_step):
    """Whole-job units per second under weak scaling: every rank processes
    units_per_rank units per step."""
    return world * units_per_rank / (ms_per_step * 1e-3)


def run_reference(args, scene):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cores = _host_cores()
    chunk = scene.n_points  # one step = one pass over the whole frame, split over the cores
    res = _run_replicas(cores, scene.seed, steps=args.warmup + args.steps, chunk=chunk)
    per_step = [max(r[3][i] for r in res) for i in range(args.warmup, args.warmup + args.steps)]
    total = sum(per_step)
    value = chunk * scene.spp * len(per_step) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(per_step),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(scene),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"the whole frame ({chunk} points) per step, split over {cores} "
                                       "oracle processes (one per host core, each with its own grid), "
                                       "oracle sample+Eq.1+Eq.2+split-collapse; step time = slowest process"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def batched_measure(n_scenes, scale, steps, warmup, scene_by_scene=True):
    """Many uneven scenes in one persistent launch per stage, replayed as a
    CUDA graph; the tile size and occupancy come from the autotuner. Also
    times the same pass issued scene by scene through the single-grid calls."""
    import torch
    from paper_1911_10217_gb300 import rll, scenes
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    ctx = rll.Context(0, stream)
    t0 = time.perf_counter()
    sc = scenes.batched_scenes(n_scenes=n_scenes, scale=scale)
    gen_s = time.perf_counter() - t0
    objs = []
    for s in sc:
        T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
        d = dict(tri=T(s.tris.reshape(-1, 9)), em=T(s.emission), boxes=T(s.boxes), pos=T(s.pos), nrm=T(s.nrm),
                 alb=T(s.albedo))
        tree = rll.Tree(ctx, d["tri"], d["em"])
        g = s.grid
        grid = rll.Grid(ctx, tree, rll.grid_params_for(g))
        objs.append(dict(s=s, d=d, tree=tree, grid=grid, rgb=torch.zeros(3, s.n_points, device=dev)))
    items = [dict(grid=o["grid"], tree=o["tree"], pos=o["d"]["pos"], nrm=o["d"]["nrm"], albedo=o["d"]["alb"],
                  boxes=o["d"]["boxes"], seed=o["s"].seed, frame=0, spp=o["s"].spp, rgb=o["rgb"]) for o in objs]
    batch = rll.Batch(ctx, items)
    tile, minb = batch.tune()
    batch.capture(do_split=True)
    for _ in range(warmup):
        batch.launch()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in ev:
        e0.record(stream)
        batch.launch()
        e1.record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    samples = sum(o["s"].n_points * o["s"].spp for o in objs)
    seq_ms = None
    if scene_by_scene:  # the same pass issued scene by scene
        key = torch.empty(max(o["s"].n_points * o["s"].spp for o in objs), dtype=torch.int32, device=dev)
        val = torch.empty_like(key, dtype=torch.float32)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for o in objs:
            s, d = o["s"], o["d"]
            n = s.n_points * s.spp
            rll.sample_and_shade(ctx, o["grid"], o["tree"], d["pos"], d["nrm"], d["alb"], d["boxes"], s.seed, 10**6,
                                 s.spp, o["rgb"], key[:n], val[:n])
            rll.learn_update_split(ctx, o["grid"], o["tree"], key[:n], val[:n])
        e1.record(stream)
        torch.cuda.synchronize()
        seq_ms = e0.elapsed_time(e1)
    status = ctx.sync_status()
    out = {"value": samples / (statistics.mean(ms) * 1e-3), "ms_per_step": statistics.mean(ms),
           "p99_ms": float(np.percentile(ms, 99)), "steps": steps, "warmup": warmup,
           "config": {"workload": f"{len(sc)} uneven scenes in one persistent launch per stage, CUDA graph replay",
                      "scenes": len(sc), "scale": scale, "samples_per_step": samples,
                      "lights_total": sum(o["s"].n_lights for o in objs),
                      "cut_sizes": sorted(set(o["s"].grid.cut_size for o in objs)),
                      "tuned_tile_points": tile, "tuned_min_blocks": minb},
           "scene_by_scene_ms": seq_ms,
           "speedup_vs_scene_by_scene": (seq_ms / statistics.mean(ms)) if seq_ms else None,
           "generation_s": gen_s, "device_status": status}
    batch.close()
    for o in objs:
        o["grid"].close()
        o["tree"].close()
    return out


def run_batched(args):
    """The batched workload on its own line."""
    r = batched_measure(args.batched_scenes, args.batched_scale, args.steps, args.warmup)
    line = {"metric": METRIC, "workload": "batched", "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic", **r}
    print(json.dumps(line))
    return 0


def serving_measure(n_sessions, frames, scale=1.0, load=0.7, budget_gb=80.0, seed=11):
    """Continuous batching of frame requests from many sessions (half of the
    frame-scale shape, half of the 4K / 1M-light shape, BF16 tables), Poisson
    arrivals at a fixed fraction of the measured capacity, admission by an HBM
    budget. Returns served samples per second, p50 / p99 frame latency and the
    device overlap of the two launch slots."""
    import torch
    from paper_1911_10217_gb300 import rll, scenes, serving
    dev = torch.device("cuda:0")
    sc = scale
    t0 = time.perf_counter()
    shape_a = scenes.frame_scene(seed=1, width=int(1920 * sc), height=int(1080 * sc))
    shape_b = scenes.dynamic_scene(seed=2, width=int(3840 * sc), height=int(2160 * sc))
    gen_s = time.perf_counter() - t0
    prec = "bf16"
    shapes = {sid: (shape_a if sid % 2 == 0 else shape_b) for sid in range(n_sessions)}
    max_items, max_records, max_cells = 64, 1 << 26, (1 << 26) - 1
    ex = serving.GpuExecutor(torch, rll, dev, max_items, max_records, max_cells, timeline=True)
    budget = int(budget_gb * 1e9)
    sched = serving.Scheduler(budget, max_items, max_records, max_cells,
                              reserved_bytes=ex.reserved_bytes(max_records, max_cells))

    def size(s):
        return serving.session_bytes(s.n_lights, s.n_points, s.grid.table_size, s.grid.cut_size, prec)

    # capacity: full launches of one session of each shape, repeated
    cal = {10**6: shape_a, 10**6 + 1: shape_b}
    for sid, s in cal.items():
        ex.create(sid, s, prec, seed=sid)
    items_sched = serving.Scheduler(10**15, max_items, max_records, max_cells)
    for sid, s in cal.items():
        items_sched.add_session(sid, 0, s.n_points * s.spp, s.grid.table_size, 10)
    items_sched.admit()
    cal_samples, t_cal = 0, 0.0
    for f in range(8):
        for sid in cal:
            items_sched.arrive(serving.Request(sid, f, 0.0))
        batch = items_sched.form_batch()
        torch.cuda.synchronize()
        c0 = time.perf_counter()
        ex.launch(0, batch, {r.session: f for r in batch})
        while not ex.poll():
            pass
        dt = time.perf_counter() - c0
        items_sched.complete(batch, 0.0)
        if f >= 2:
            t_cal += dt
            cal_samples += sum(cal[r.session].n_points * cal[r.session].spp for r in batch)
    for sid in cal:
        ex.release(sid)
    ex.timeline.clear()
    capacity = cal_samples / t_cal
    mean_samples = np.mean([shapes[s].n_points * shapes[s].spp for s in shapes])
    rate_total = load * capacity / mean_samples   # frames per second
    rng = np.random.default_rng(seed)
    arrivals = {sid: serving.poisson_arrivals(rng, frames, rate_total / n_sessions) for sid in shapes}
    for sid, s in shapes.items():
        sched.add_session(sid, size(s), s.n_points * s.spp, s.grid.table_size, frames)
    # each session its own Philox seed
    orig_create = ex.create
    ex.create = lambda sid, s, p: orig_create(sid, s, p, seed=1000 + sid)
    w0 = time.perf_counter()
    log = serving.serve(ex, sched, shapes, arrivals, precision=prec, timeout_s=3600.0)
    wall = time.perf_counter() - w0
    spans = ex.device_intervals()
    lat = np.array([1e3 * (r.done - r.arrival) for r in log])
    starts = {}
    for r in log:
        starts.setdefault(r.start, []).append(r)
    served = sum(shapes[r.session].n_points * shapes[r.session].spp for r in log)
    # launches of the two slots on the device at the same time
    ends = {}
    for slot, a, b in spans:
        ends.setdefault(slot, []).append((a, b))
    overlap = sum(1 for a1, b1 in ends.get(0, []) for a2, b2 in ends.get(1, []) if a1 < b2 and a2 < b1)
    return {"value": served / wall, "p50_frame_ms": float(np.percentile(lat, 50)),
            "p99_frame_ms": float(np.percentile(lat, 99)), "frames": len(log), "launches": len(starts),
            "mean_sessions_per_launch": len(log) / len(starts), "offered_load_fraction": load,
            "capacity_samples_per_s": capacity, "overlapping_launch_pairs": overlap,
            "sessions": n_sessions, "frames_per_session": frames,
            "shape_a": f"{shape_a.width}x{shape_a.height}, {shape_a.n_lights} lights, M={shape_a.grid.cut_size}",
            "shape_b": f"{shape_b.width}x{shape_b.height}, {shape_b.n_lights} lights, M={shape_b.grid.cut_size}",
            "budget_gb": budget_gb, "table_precision": prec,
            "resident_gb": sum(size(s) for s in shapes.values()) / 1e9,
            "wall_s": wall, "generation_s": gen_s, "device_status": ex.status()}


def run_serving(args):
    """The serving workload on its own line (64 sessions by default)."""
    r = serving_measure(args.serving_sessions, args.serving_frames, args.serving_scale, args.serving_load,
                        args.serving_budget_gb)
    line = {"metric": METRIC, "workload": "serving", "value": r["value"], "unit": UNIT, "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32 arithmetic, bf16 tables", "data": "synthetic",
            "p50_frame_ms": r["p50_frame_ms"], "p99_frame_ms": r["p99_frame_ms"],
            "config": {"workload": f"{r['sessions']} sessions, continuous batching, HBM-budget admission",
                       **{k: r[k] for k in ("sessions", "frames_per_session", "shape_a", "shape_b", "budget_gb",
                                            "table_precision", "resident_gb")}},
            **{k: r[k] for k in ("frames", "launches", "mean_sessions_per_launch", "offered_load_fraction",
                                 "capacity_samples_per_s", "overlapping_launch_pairs", "wall_s", "generation_s",
                                 "device_status")}}
    print(json.dumps(line))
    return 0


def dynamic_measure(frames, precisions, scale=1.0, mse=True):
    """Dynamic lighting (1M triangles, 10% blinking, 3840x2160, M = 64,
    split-collapse every frame) per table precision: sampling and learning
    time per frame (frames 3.. of a fresh grid), touched cells, the learning
    step's algorithmic bytes, and optionally the 1-spp MSE against a
    high-spp energy-sampler reference of the last frame."""
    import torch
    from paper_1911_10217_gb300 import rll, scenes
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    ctx = rll.Context(0, stream)
    s = scenes.dynamic_scene(width=int(3840 * scale), height=int(2160 * scale))
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    tri, bound, em0 = T(s.tris.reshape(-1, 9)), T(s.emission_bound()), T(s.emission)
    omega, phase = T(s.blink_omega), T(s.blink_phase)
    mask = T(s.blink_mask.astype(np.float32))
    boxes, pos, nrm, alb = T(s.boxes), T(s.pos), T(s.nrm), T(s.albedo)
    tree = rll.Tree(ctx, tri, bound)
    P = s.n_points
    em = torch.empty_like(em0)

    def set_emission(frame):
        t = frame / 30.0
        sc = 1.0 + mask * 0.9 * torch.sin(omega * t + phase)
        torch.mul(em0, sc[:, None], out=em)
        tree.update_emission(em)

    rgb = torch.empty(3, P, device=dev)
    key = torch.empty(P * s.spp, dtype=torch.int32, device=dev)
    val = torch.empty(P * s.spp, device=dev)
    g = s.grid
    results = {}
    for prec in precisions:
        grid = rll.Grid(ctx, tree, rll.grid_params_for(g, precision=prec))
        ms, touched = [], []
        for f in range(frames):
            set_emission(f)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            rll.sample_and_shade(ctx, grid, tree, pos, nrm, alb, boxes, s.seed, f, s.spp, rgb, key, val)
            e1.record(stream)
            rll.learn_update_split(ctx, grid, tree, key, val)
            e2.record(stream)
            ms.append((e0, e1, e2))
            if f >= 3 and (f % 8 == 3 or f == frames - 1):  # outside the event pairs: a host round trip only
                touched.append(grid.touched_cells())
        torch.cuda.synchronize()
        t = [a.elapsed_time(c) for a, b, c in ms][3:]
        t_s = [a.elapsed_time(b) for a, b, c in ms][3:]
        t_l = [b.elapsed_time(c) for a, b, c in ms][3:]
        n_touched = statistics.mean(touched) if touched else float("nan")
        e = 4 if prec == "fp32" else 2
        lb = learn_step_bytes(P * s.spp, n_touched, g.cut_size, prec)
        r = {"ms_per_frame": statistics.mean(t), "p99_frame_ms": float(np.percentile(t, 99)),
             "sample_ms": statistics.mean(t_s), "learn_update_split_ms": statistics.mean(t_l),
             "touched_cells_per_frame": n_touched,
             "learn_algorithmic_bytes_per_frame": lb,
             "learn_algorithmic_gbs": lb / (statistics.mean(t_l) * 1e-3) / 1e9,
             "samples_per_s": P * s.spp / (statistics.mean(t) * 1e-3),
             "table_bytes": g.table_size * g.cut_size * (4 + 2 * e)}
        if mse:
            # reference of the last frame: energy sampler, 256 spp
            set_emission(frames - 1)
            ref = torch.zeros(3, P, device=dev, dtype=torch.float64)
            tmp = torch.empty(3, P, device=dev)
            for i in range(32):
                rll.sample_power(ctx, tree, pos, nrm, alb, boxes, 9999, 200000 + i, 8, tmp)
                ref += tmp.double()
            ref /= 32
            rll.sample_and_shade(ctx, grid, tree, pos, nrm, alb, boxes, 4242, 300000, 1, tmp)
            err = float(((tmp.double() - ref) ** 2).mean())
            rll.sample_power(ctx, tree, pos, nrm, alb, boxes, 4242, 300000, 1, tmp)
            err_pow = float(((tmp.double() - ref) ** 2).mean())
            r.update({"mse_1spp": err, "energy_sampler_mse_1spp": err_pow, "mse_ratio_vs_energy": err_pow / err})
        results[prec] = r
        grid.close()
    config = {"workload": "dynamic lighting, 10% blinking lights, split-collapse every frame",
              "points": P, "lights": s.n_lights, "cut_size": g.cut_size, "table_size": g.table_size,
              "frames": frames, "timed_frames": f"3..{frames - 1} of a fresh grid", "boxes": int(s.boxes.shape[0])}
    return config, results, ctx.sync_status()


def run_dynamic(args):
    config, results, status = dynamic_measure(args.dynamic_frames, args.dynamic_precisions.split(","),
                                              args.dynamic_scale)
    line = {"metric": METRIC, "workload": "dynamic", "unit": UNIT, "n_gpus": 1, "data": "synthetic",
            "config": config, "precisions": results, "device_status": status}
    print(json.dumps(line))
    return 0


def leaf_spread(grid):
    """How unequal the learned leaf weights of the occupied cells are: mean
    over cells of max Q / mean Q of the cut's leaves (1 = all equal)."""
    st = grid.export()
    occ = st["keys"] != np.uint64(0xFFFFFFFFFFFFFFFF)
    q = st["q"][occ, :grid.m].astype(np.float64)
    r = q.max(axis=1) / np.maximum(q.mean(axis=1), 1e-300)
    return {"cells": int(occ.sum()), "mean_max_over_mean": float(r.mean()),
            "median_max_over_mean": float(np.median(r))}


def run_split(args):
    """Iterated split-collapse: the frame workload learned for a number of
    passes with split-collapse repeated up to K steps per cell and pass, for
    several K; per K the pass time (split-collapse separately), how far the
    cuts have equalised the leaf weights after 1, 4, 16, ... passes, and the
    1-spp MSE at the end."""
    import torch
    from paper_1911_10217_gb300 import rll, scenes
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    ctx = rll.Context(0, stream)
    s = scenes.frame_scene()
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    tri, em, boxes = T(s.tris.reshape(-1, 9)), T(s.emission), T(s.boxes)
    pos, nrm, alb = T(s.pos), T(s.nrm), T(s.albedo)
    tree = rll.Tree(ctx, tri, em)
    P = s.n_points
    rgb = torch.empty(3, P, device=dev)
    key = torch.empty(P, dtype=torch.int32, device=dev)
    val = torch.empty(P, device=dev)
    checkpoints = {1, 4, 16, 64, 256, 1024}
    results = {}
    for K in [int(k) for k in args.split_sweep.split(",")]:
        grid = rll.Grid(ctx, tree, rll.grid_params_for(s.grid, split_iterations=K))
        ev, spread = [], {}
        for f in range(args.split_passes):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            rll.sample_and_shade(ctx, grid, tree, pos, nrm, alb, boxes, s.seed, f, 1, rgb, key, val)
            rll.learn_update(ctx, grid, key, val)
            e[1].record(stream)
            rll.split_collapse(ctx, grid, tree)
            e[2].record(stream)
            ev.append(e)
            if f + 1 in checkpoints:
                torch.cuda.synchronize()
                spread[f + 1] = leaf_spread(grid)
        torch.cuda.synchronize()
        t_pass = [a.elapsed_time(c) for a, _, c in ev][3:]
        t_split = [b.elapsed_time(c) for _, b, c in ev][3:]
        results[K] = {"ms_per_pass": statistics.mean(t_pass), "split_ms": statistics.mean(t_split),
                      "samples_per_s": P / (statistics.mean(t_pass) * 1e-3), "leaf_spread": spread,
                      "mse_equal_spp": quality(rll, ctx, grid, tree, s, pos, nrm, alb, boxes, dev)}
        grid.close()
    line = {"metric": METRIC, "workload": "split", "unit": UNIT, "n_gpus": 1, "data": "synthetic",
            "config": dict(workload_config(s), split_iterations="swept", passes=args.split_passes),
            "split_iterations": results, "device_status": ctx.sync_status()}
    print(json.dumps(line))
    return 0


def run_sky(args):
    """Sky-dome interior (the situation of the paper's "Arch interior" scene,
    Section 4): a closed room lit through small windows and skylights by a
    2048-triangle sky dome and a small bright distant quad; 1920 x 1080 floor
    points (--sky-sun 1 adds a small bright distant quad for a directional
    light). For each combination of the swept in-cluster modes, learning
    rates, floors, cut sizes, split thresholds and reward modes: learns for
    --sky-passes passes (each timed: sample + Eq. 1/2 + split-collapse), then
    reports the MSE of the learned sampler and of the energy sampler at 1, 4
    and 8 spp against a common reference (the energy sampler at
    --sky-ref-spp spp), and the MSE of a fresh grid at 1 spp."""
    import torch
    from paper_1911_10217_gb300 import rll, scenes
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    ctx = rll.Context(0, stream)
    s = scenes.sky_scene(sun=bool(args.sky_sun))
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    tri, em, boxes = T(s.tris.reshape(-1, 9)), T(s.emission), T(s.boxes)
    pos, nrm, alb = T(s.pos), T(s.nrm), T(s.albedo)
    tree = rll.Tree(ctx, tri, em)
    P = s.n_points
    rgb = torch.empty(3, P, device=dev)
    key = torch.empty(P, dtype=torch.int32, device=dev)
    val = torch.empty(P, device=dev)
    ref = torch.zeros(3, P, device=dev, dtype=torch.float64)
    batches = max(1, args.sky_ref_spp // 32)
    for i in range(batches):
        rll.sample_power(ctx, tree, pos, nrm, alb, boxes, 4242, 200000 + i, 32, rgb)
        ref += rgb.double()
    ref /= batches

    def mse_of(fn, spp, reps=4):
        acc = 0.0
        for r in range(reps):
            fn(spp, 70000 + 17 * r)
            acc += float(((rgb.double() - ref) ** 2).mean())
        return acc / reps

    def power_pass(spp, frame):
        rll.sample_power(ctx, tree, pos, nrm, alb, boxes, 31337, frame, spp, rgb)

    energy = {f"{spp}spp": mse_of(power_pass, spp) for spp in (1, 4, 8)}
    runs = []
    combos = [(mode, float(a), float(e), int(m), float(t), rw) for mode in args.sky_modes.split(",")
              for a in args.sky_alphas.split(",") for e in args.sky_eps.split(",")
              for m in args.sky_cuts.split(",") for t in args.sky_thresholds.split(",")
              for rw in args.sky_rewards.split(",")]
    for mode, alpha, eps, cut, thr, reward in combos:
        if True:
            params = rll.grid_params_for(s.grid, mode=mode, alpha=alpha, eps=eps, cut_size=cut, threshold=thr,
                                         reward=reward)
            grid = rll.Grid(ctx, tree, params)
            fresh = rll.Grid(ctx, tree, params)
            ev = []
            for f in range(args.sky_passes):
                e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                e[0].record(stream)
                rll.sample_and_shade(ctx, grid, tree, pos, nrm, alb, boxes, s.seed, f, 1, rgb, key, val)
                rll.learn_update_split(ctx, grid, tree, key, val)
                e[1].record(stream)
                ev.append(e)
            torch.cuda.synchronize()
            t_pass = [x.elapsed_time(y) for x, y in ev][3:]

            def rll_pass(spp, frame, g=grid):
                rll.sample_and_shade(ctx, g, tree, pos, nrm, alb, boxes, 31337, frame, spp, rgb)

            mse = {}
            for spp in (1, 4, 8):
                m = mse_of(rll_pass, spp)
                mse[f"{spp}spp"] = {"rll": m, "energy_sampler": energy[f"{spp}spp"],
                                    "energy_over_rll": energy[f"{spp}spp"] / m}
            mse["fresh_grid_1spp"] = mse_of(lambda k, fr: rll_pass(k, fr, fresh), 1, reps=2)
            runs.append({"in_cluster": mode, "alpha": alpha, "eps": eps, "cut_size": cut, "threshold": thr,
                         "reward": reward,
                         "ms_per_pass": statistics.mean(t_pass),
                         "samples_per_s": P / (statistics.mean(t_pass) * 1e-3), "mse": mse})
            grid.close()
            fresh.close()
    line = {"metric": METRIC, "workload": "sky", "unit": UNIT, "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "sky-dome interior, 1920x1080 floor points, 2048 dome triangles"
                                   + (" + 2 sun triangles" if args.sky_sun else "") + ", "
                                   f"{int(s.boxes.shape[0])} occluder boxes (walls with 16 windows, 2 skylights), "
                                   "one learning pass per step", "points": P, "lights": s.n_lights,
                       "boxes": int(s.boxes.shape[0]), "cut_size": s.grid.cut_size,
                       "table_size": s.grid.table_size, "cell_size": s.grid.cell_size, "passes": args.sky_passes},
            "runs": runs, "reference": f"energy sampler, {batches * 32} spp",
            "device_status": ctx.sync_status()}
    print(json.dumps(line))
    return 0


def run_paths(args):
    """Path vertices with footprint-sized cells (Section 3: cells sized from
    the ray footprint of each path vertex, coarser on later bounces): the
    frame workload's 1920 x 1080 primary points (finest level) and one diffuse
    bounce vertex each, footprint (N_t p_A)^(-1/2) for each N_t of
    --paths-tiles. For each N_t a grid of --paths-levels levels, and once a
    single-level grid, learn for --paths-passes passes; the pass time, the
    cells per level and the 1-spp MSE at the primary and at the bounce
    vertices after each of --paths-checkpoints passes are reported, beside
    the energy sampler, against the energy sampler at --paths-ref-spp spp."""
    import torch
    from paper_1911_10217_gb300 import rll, scenes
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    ctx = rll.Context(0, stream)
    base = scenes.frame_scene()
    s = scenes.path_scene(base, levels=args.paths_levels, paths_per_tile=1.0)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    tri, em, boxes = T(s.tris.reshape(-1, 9)), T(s.emission), T(s.boxes)
    # the bounce vertices by the library: one diffuse bounce from every primary point
    P0 = base.n_points
    P = 2 * P0
    pos, nrm = torch.empty(3, P, device=dev), torch.empty(3, P, device=dev)
    fp1 = torch.empty(P, device=dev)
    pos[:, :P0], nrm[:, :P0], fp1[:P0] = T(base.pos), T(base.nrm), T(s.footprint)
    b = s.bounce
    by, bn, bf = torch.empty(3, P0, device=dev), torch.empty(3, P0, device=dev), torch.empty(P0, device=dev)
    rll.bounce_vertices(ctx, pos[:, :P0].contiguous(), nrm[:, :P0].contiguous(), boxes, b.room, b.seed, b.frame,
                        b.paths_per_tile, by, bn, bf)
    pos[:, P0:], nrm[:, P0:], fp1[P0:] = by, bn, bf
    alb = torch.cat([T(base.albedo), T(b.albedo)])
    tree = rll.Tree(ctx, tri, em)
    rgb = torch.empty(3, P, device=dev)
    key = torch.empty(P, dtype=torch.int32, device=dev)
    val = torch.empty(P, device=dev)
    ref = torch.zeros(3, P, device=dev, dtype=torch.float64)
    batches = max(1, args.paths_ref_spp // 32)
    for i in range(batches):
        rll.sample_power(ctx, tree, pos, nrm, alb, boxes, 4242, 300000 + i, 32, rgb)
        ref += rgb.double()
    ref /= batches

    def mse_split(fn, reps=2):
        a = b = 0.0
        for r in range(reps):
            fn(80000 + 13 * r)
            e = (rgb.double() - ref) ** 2
            a += float(e[:, :P0].mean())
            b += float(e[:, P0:].mean())
        return {"primary": a / reps, "bounce": b / reps}

    out = {"energy_sampler_mse_1spp": mse_split(
        lambda fr: rll.sample_power(ctx, tree, pos, nrm, alb, boxes, 31337, fr, 1, rgb))}
    checkpoints = sorted(int(c) for c in args.paths_checkpoints.split(","))
    configs = [("single_level", 1, 1 << 20, None, None)]
    for nt in (float(x) for x in args.paths_tiles.split(",")):
        fp = fp1.clone()
        fp[P0:] /= float(np.sqrt(nt))
        configs.append((f"levels{args.paths_levels}_Nt{nt:g}", args.paths_levels, args.paths_table, fp, nt))
    for name, levels, table, fp, nt in configs:
        grid = rll.Grid(ctx, tree, rll.grid_params_for(s.grid, levels=levels, table_size=table))
        ev, curve = [], {}
        for f in range(checkpoints[-1]):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e[0].record(stream)
            rll.sample_and_shade(ctx, grid, tree, pos, nrm, alb, boxes, s.seed, f, 1, rgb, key, val, footprint=fp)
            rll.learn_update_split(ctx, grid, tree, key, val)
            e[1].record(stream)
            ev.append(e)
            if f + 1 in checkpoints:
                curve[f + 1] = mse_split(lambda fr, g=grid, fa=fp: rll.sample_and_shade(
                    ctx, g, tree, pos, nrm, alb, boxes, 31337, fr, 1, rgb, footprint=fa))
        torch.cuda.synchronize()
        t = [x.elapsed_time(y) for x, y in ev[3:]]
        st = grid.export()
        occ = st["keys"] != np.uint64(0xFFFFFFFFFFFFFFFF)
        cells = np.bincount(np.nonzero(occ)[0] // table, minlength=levels).tolist()
        last = curve[checkpoints[-1]]
        out[name] = {"levels": levels, "paths_per_tile": nt, "table_size_per_level": table,
                     "ms_per_pass": statistics.median(t), "samples_per_s": P / (statistics.median(t) * 1e-3),
                     "cells_per_level": cells, "mse_1spp_after_passes": curve,
                     "energy_over_rll_at_end": {k: out["energy_sampler_mse_1spp"][k] / last[k] for k in last}}
        grid.close()
    line = {"metric": METRIC, "workload": "paths", "unit": UNIT, "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "frame-scale scene, 1920x1080 primary points + one diffuse bounce vertex each, "
                                   "footprint-sized cells", "points": P, "primary_points": P0,
                       "lights": s.n_lights, "boxes": int(s.boxes.shape[0]), "cut_size": s.grid.cut_size,
                       "cell_size": s.grid.cell_size, "passes": checkpoints[-1]},
            "results": out, "reference": f"energy sampler, {batches * 32} spp", "device_status": ctx.sync_status()}
    print(json.dumps(line))
    return 0


def run_trees(args):
    """Light-tree builders at equal cost: for the frame workload and the sky
    interior, the radix tree of the Morton codes (Section 3.1), the
    surface-area-orientation split positions and the median split positions;
    per builder the leaf depth, the pass time (sampling, learning,
    split-collapse) over --trees-passes learning passes, and the 1-spp MSE
    after them (mean of --trees-frames frames) against
    the energy sampler at 1024 spp (the energy sampler uses the same light
    order for every tree)."""
    import torch
    from paper_1911_10217_gb300 import rll, scenes
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    ctx = rll.Context(0, stream)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    results = {}
    for sname, s in (("frame", scenes.frame_scene()), ("sky", scenes.sky_scene())):
        tri, em, boxes = T(s.tris.reshape(-1, 9)), T(s.emission), T(s.boxes)
        pos, nrm, alb = T(s.pos), T(s.nrm), T(s.albedo)
        P = s.n_points
        rgb = torch.empty(3, P, device=dev)
        key = torch.empty(P, dtype=torch.int32, device=dev)
        val = torch.empty(P, device=dev)
        ref = torch.zeros(3, P, device=dev, dtype=torch.float64)
        tree0 = rll.Tree(ctx, tri, em)
        for i in range(32):
            rll.sample_power(ctx, tree0, pos, nrm, alb, boxes, 4242, 400000 + i, 32, rgb)
            ref += rgb.double()
        ref /= 32
        alpha = s.grid.alpha if sname == "frame" else 0.01
        for builder in args.trees_builders.split(","):
            tree = tree0 if builder == "lbvh" else rll.Tree(ctx, tri, em, builder=builder)
            ex = tree.export()
            n = tree.n
            stack, d = [0], {0: 0}
            while stack:
                v = stack.pop()
                if v < n - 1:
                    for c in (ex["left"][v], ex["right"][v]):
                        d[int(c)] = d[v] + 1
                        stack.append(int(c))
            leaf_depth = np.array([d[n - 1 + l] for l in range(n)])
            grid = rll.Grid(ctx, tree, rll.grid_params_for(s.grid, alpha=alpha))
            ev = []
            for f in range(args.trees_passes):
                e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
                e[0].record(stream)
                rll.sample_and_shade(ctx, grid, tree, pos, nrm, alb, boxes, s.seed, f, 1, rgb, key, val)
                e[1].record(stream)
                rll.learn_update(ctx, grid, key, val)
                e[2].record(stream)
                rll.split_collapse(ctx, grid, tree)
                e[3].record(stream)
                ev.append(e)
            torch.cuda.synchronize()
            tim = [[e[i].elapsed_time(e[i + 1]) for i in range(3)] for e in ev[3:]]
            mse = []
            for r in range(args.trees_frames):
                rll.sample_and_shade(ctx, grid, tree, pos, nrm, alb, boxes, 31337, 90000 + r, 1, rgb)
                mse.append(float(((rgb.double() - ref) ** 2).mean()))
            rll.sample_power(ctx, tree, pos, nrm, alb, boxes, 31337, 90000, 1, rgb)
            mse_pow = float(((rgb.double() - ref) ** 2).mean())
            results[f"{sname}/{builder}"] = {
                "leaf_depth_mean": float(leaf_depth.mean()), "leaf_depth_max": int(leaf_depth.max()),
                "ms_sample": statistics.mean(t[0] for t in tim), "ms_learn": statistics.mean(t[1] for t in tim),
                "ms_split": statistics.mean(t[2] for t in tim), "mse_1spp_mean": statistics.mean(mse),
                "mse_1spp_runs": mse, "energy_sampler_mse_1spp": mse_pow,
                "energy_over_rll": mse_pow / statistics.mean(mse), "alpha": alpha}
            grid.close()
    print(json.dumps({"metric": METRIC, "workload": "trees", "unit": UNIT, "n_gpus": 1, "data": "synthetic",
                      "passes": args.trees_passes, "results": results, "reference": "energy sampler, 1024 spp",
                      "device_status": ctx.sync_status()}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=29)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-quality", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-workload-extras", action="store_true",
                    help="skip the 4K dynamic-lighting and short serving figures of the default line")
    ap.add_argument("--sample-min-blocks", type=int, default=4)
    ap.add_argument("--separate-split", action="store_true",
                    help="learning step as rll_learn_update + rll_split_collapse instead of the fused call")
    ap.add_argument("--host-chunks", type=int, default=8,
                    help="chunks of the host-buffer pass (copy/compute overlap)")
    ap.add_argument("--tree", default="lbvh", choices=["lbvh", "saoh", "median"])
    ap.add_argument("--trees-builders", default="lbvh,saoh,median")
    ap.add_argument("--trees-frames", type=int, default=16)
    ap.add_argument("--mode", default="descent", choices=["descent", "descent2", "uniform"])
    ap.add_argument("--workload", default="frame",
                    choices=["frame", "batched", "serving", "dynamic", "split", "sky", "paths", "trees"])
    ap.add_argument("--trees-passes", type=int, default=256)
    ap.add_argument("--paths-checkpoints", default="1,4,16,64,128")
    ap.add_argument("--paths-tiles", default="100,1000")
    ap.add_argument("--paths-levels", type=int, default=8)
    ap.add_argument("--paths-table", type=int, default=1 << 19)
    ap.add_argument("--paths-ref-spp", type=int, default=1024)
    ap.add_argument("--sky-passes", type=int, default=256)
    ap.add_argument("--sky-modes", default="descent")
    ap.add_argument("--sky-alphas", default="0.003,0.01,0.03")
    ap.add_argument("--sky-ref-spp", type=int, default=4096)
    ap.add_argument("--sky-sun", type=int, default=0, choices=[0, 1])
    ap.add_argument("--sky-eps", default="0.02")
    ap.add_argument("--sky-cuts", default="32,128")
    ap.add_argument("--sky-thresholds", default="2")
    ap.add_argument("--sky-rewards", default="cluster")
    ap.add_argument("--split-iterations", type=int, default=1)
    ap.add_argument("--split-sweep", default="1,2,4,16,64")
    ap.add_argument("--split-passes", type=int, default=64)
    ap.add_argument("--dynamic-scale", type=float, default=1.0)
    ap.add_argument("--dynamic-frames", type=int, default=120)
    ap.add_argument("--dynamic-precisions", default="fp32,fp16,bf16")
    ap.add_argument("--serving-sessions", type=int, default=64)
    ap.add_argument("--serving-frames", type=int, default=160)
    ap.add_argument("--serving-scale", type=float, default=1.0)
    ap.add_argument("--serving-load", type=float, default=0.7)
    ap.add_argument("--serving-budget-gb", type=float, default=80.0)
    ap.add_argument("--batched-scenes", type=int, default=256)
    ap.add_argument("--batched-scale", type=float, default=1.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "dynamic":
        return run_dynamic(args)
    if args.workload == "sky":
        return run_sky(args)
    if args.workload == "paths":
        return run_paths(args)
    if args.workload == "trees":
        return run_trees(args)
    if args.workload == "split":
        return run_split(args)
    from paper_1911_10217_gb300 import scenes
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    scene = scenes.frame_scene(seed=1 + rank)
    scene.grid.split_iterations = args.split_iterations
    if args.impl == "reference":
        return run_reference(args, scene)

    import torch
    from paper_1911_10217_gb300 import rll

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = rll.Context(local, stream)
    ctx.set_option("sample_min_blocks", args.sample_min_blocks)
    ctx.set_option("host_chunks", args.host_chunks)

    def T(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    tri, em, boxes = T(scene.tris.reshape(-1, 9)), T(scene.emission), T(scene.boxes)
    pos, nrm, alb = T(scene.pos), T(scene.nrm), T(scene.albedo)
    P, S = scene.n_points, scene.spp
    tree = rll.Tree(ctx, tri, em, builder=args.tree)
    g = scene.grid
    params = rll.grid_params_for(g, mode=args.mode)
    grid = rll.Grid(ctx, tree, params)
    rgb = torch.empty(3, P, device=dev)
    key = torch.empty(P * S, dtype=torch.int32, device=dev)
    val = torch.empty(P * S, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(frame, ev=None):
        if ev:
            ev[0].record(stream)
        rll.sample_and_shade(ctx, grid, tree, pos, nrm, alb, boxes, scene.seed, frame, S, rgb, key, val)
        if ev:
            ev[1].record(stream)
        if args.separate_split:
            rll.learn_update(ctx, grid, key, val)
            if ev:
                ev[2].record(stream)
            rll.split_collapse(ctx, grid, tree)
        else:  # Eq. 1, split-collapse and Eq. 2 in the learning kernels
            rll.learn_update_split(ctx, grid, tree, key, val)
            if ev:
                ev[2].record(stream)
        if ev:
            ev[3].record(stream)

    frame = 0
    for _ in range(args.warmup):
        step(frame)
        frame += 1
    torch.cuda.synchronize()
    if ctx.sync_status() != 0:
        raise RuntimeError("device status raised during warm-up")

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        step(frame, evs[i])
        frame += 1
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    status = ctx.sync_status()
    n_touched = grid.touched_cells()  # cells the last timed pass learned
    t_sample = [e[0].elapsed_time(e[1]) for e in evs]
    t_learn = [e[1].elapsed_time(e[2]) for e in evs]
    t_split = [e[2].elapsed_time(e[3]) for e in evs]
    t_step = [e[0].elapsed_time(e[3]) for e in evs]
    total_ms = max_over_ranks(sum(t_step), dist, dev)
    ms_step = total_ms / args.steps
    value = job_throughput(world, P * S, ms_step)

    # ---- end to end through the host-buffer entry point (pinned host memory)
    hpos = torch.from_numpy(np.ascontiguousarray(scene.pos)).pin_memory()
    hnrm = torch.from_numpy(np.ascontiguousarray(scene.nrm)).pin_memory()
    halb = torch.from_numpy(np.ascontiguousarray(scene.albedo)).pin_memory()
    hbox = torch.from_numpy(np.ascontiguousarray(scene.boxes)).pin_memory()
    hrgb = torch.empty(3, P, dtype=torch.float32).pin_memory()
    for _ in range(0 if args.no_e2e else 2):
        rll.render_pass_host(ctx, grid, tree, hpos, hnrm, halb, hbox, scene.seed, frame, S, hrgb)
        frame += 1
    e2e_ms = [float("nan")]
    for _ in range(0 if args.no_e2e else max(3, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rll.render_pass_host(ctx, grid, tree, hpos, hnrm, halb, hbox, scene.seed, frame, S, hrgb)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        frame += 1
    e2e_ms = [t for t in e2e_ms if t == t] or [float("nan")]
    e2e_step = max_over_ranks(statistics.mean(e2e_ms), dist, dev)  # every rank runs the loop

    out = None
    if rank == 0:
        peaks, peak_kind = load_peaks()
        sm_clock = peaks.get("sm_max_mhz", 2070.0)
        alu_peak = SM_COUNT * FP32_LANES_PER_SM * sm_clock * 1e6 / 1e12  # Tops/s
        n_sample = P * S
        ops = ops_per_sample(int(scene.boxes.shape[0]), scene.n_lights, grid.m) * n_sample
        t_s = statistics.mean(t_sample) * 1e-3
        achieved = ops / t_s / 1e12
        hbm_ach = bytes_per_sample() * n_sample / t_s / 1e9
        learn_bytes = learn_step_bytes(n_sample, n_touched, grid.M)
        t_l = statistics.mean(t_learn) * 1e-3
        # our kernels per step: the box sort and sampling = 2; learning: count, claim, scatter, the warp,
        # two-warp and block paths (one launch), the sorting block path = 5; split-collapse 1 unless
        # fused into learning (an ncu launch list of the pass shows them)
        launches_per_step = 2 + 5 + (1 if args.separate_split else 0)
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": dict(workload_config(scene, args.tree, args.mode),
                              passes=f"passes {args.warmup}..{args.warmup + args.steps - 1} of a fresh grid timed "
                                     f"(passes 0..{args.warmup - 1} untimed warm-up)"),
               "roofline": {"kernel": "k_sample (sample_and_shade)", "bound": "alu",
                            "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                            "frac": achieved / alu_peak, "traffic": K_SAMPLE_DRAM_BYTES,
                            "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                            "peak_source": f"derived: {SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                                           f"{sm_clock:.0f} MHz ({peak_kind} sm_max_mhz)",
                            "ops_per_sample": ops / n_sample,
                            "hbm_achieved_gbs": hbm_ach,
                            "hbm_frac_of_measured": hbm_ach / peaks.get("hbm_gbs", 6800.0)},
               "e2e": {"value": (world * P * S / (e2e_step * 1e-3)) if e2e_step == e2e_step else None,
                       "unit": UNIT,
                       "h2d_bytes_per_step": int(28 * P + 24 * scene.boxes.shape[0]),
                       "d2h_bytes_per_step": int(12 * P)},
               "gpu_launches": args.steps * launches_per_step,
               "clocks": clk,
               "extras": {"per_kernel_ms": ({"sample_and_shade": statistics.mean(t_sample),
                                             "learn_update": statistics.mean(t_learn),
                                             "split_collapse": statistics.mean(t_split)}
                                            if args.separate_split else
                                            {"sample_and_shade": statistics.mean(t_sample),
                                             "learn_update_split": statistics.mean(t_learn)}),
                          "p50_frame_ms": statistics.median(t_step),
                          "p99_frame_ms": float(np.percentile(t_step, 99)),
                          "learn_update_algorithmic_gbs": learn_bytes / t_l / 1e9,
                          "learn_update_algorithmic_bytes": learn_bytes,
                          "touched_cells_last_pass": n_touched,
                          "wall_s_timed_region_incl_flush": wall,
                          "device_status": status}}
        if not args.no_quality:
            out["extras"]["mse_equal_spp"] = quality(rll, ctx, grid, tree, scene, pos, nrm, alb, boxes, dev)
        if not args.no_workload_extras and world == 1:
            # the 4K / 1M-light shape in binary32 and bfloat16 tables, and a short serving run
            grid.close()
            cfg, res, st = dynamic_measure(8, ["fp32", "bf16"], mse=False)
            out["extras"]["dynamic_4k"] = {"config": cfg, "precisions": res, "device_status": st}
            out["extras"]["serving"] = serving_measure(16, 64)
            # the batched form: 256 uneven scenes (166 M samples) per graph replay
            out["extras"]["batched"] = batched_measure(256, 1.0, 5, 3, scene_by_scene=False)
        if not args.no_cpu_baseline and world == 1:  # the host baseline belongs to the one-GPU line
            out["cpu_baseline"] = cpu_baseline(scene)
        print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def quality(rll, ctx, grid, tree, scene, pos, nrm, alb, boxes, dev, frames=4):
    """MSE at 1 spp of the learned sampler and of the energy-based sampler
    against a 256-spp energy-sampler reference (not timed), each the mean
    over `frames` frames (single frames are dominated by rare high-weight
    samples)."""
    import torch
    P = scene.n_points
    ref = torch.zeros(3, P, device=dev, dtype=torch.float64)
    tmp = torch.empty(3, P, device=dev)
    n_ref = 32
    for i in range(n_ref):
        rll.sample_power(ctx, tree, pos, nrm, alb, boxes, 7777, 100000 + i, 8, tmp)
        ref += tmp.double()
    ref /= n_ref
    mse_rll = mse_pow = 0.0
    for f in range(frames):
        rll.sample_and_shade(ctx, grid, tree, pos, nrm, alb, boxes, 4242, 90000 + f, 1, tmp)
        mse_rll += float(((tmp.double() - ref) ** 2).mean()) / frames
        rll.sample_power(ctx, tree, pos, nrm, alb, boxes, 4242, 90000 + f, 1, tmp)
        mse_pow += float(((tmp.double() - ref) ** 2).mean()) / frames
    return {"rll_1spp": mse_rll, "energy_sampler_1spp": mse_pow, "ratio": mse_pow / mse_rll,
            "reference": "energy sampler, 256 spp", "frames": frames}


if __name__ == "__main__":
    sys.exit(main())
