"""Continuous-batching request loop for many render sessions.

Sessions are admitted while their resident device state (light tree, hash
grid with learned cuts, G-buffer, output) fits a memory budget; a session
leaves, and frees its state, when its last frame is done. Frame requests
arrive over time; whenever one of the launch slots is free, the scheduler
forms a batch from the oldest pending requests of admitted sessions that
have no frame in flight (a session's frames depend on each other) and
launches it as one batched pass (rll_batch_*: one persistent sampling
kernel for all its scenes, one bucketing of the records, one learning
kernel). Two launch slots on two CUDA streams let a new batch start while the
previous one still runs, so requests that arrive during a launch join the
next one and its work is on the device at the same time; a launch enqueues
its descriptor upload and pass without waiting for its stream.

Each session has its own Philox seed and its own cells in the batch's
record keys, so its results do not depend on which other sessions share a
launch (tests/test_gpu_serving.py checks alone vs in the mix).

The Scheduler class holds only the policy and runs without a GPU; the
GpuExecutor class drives the CUDA library.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np


@dataclasses.dataclass
class Request:
    session: int
    frame: int
    arrival: float
    start: float = -1.0
    done: float = -1.0


@dataclasses.dataclass
class SessionState:
    sid: int
    bytes: int
    samples: int              # samples per frame
    cells: int                # hash table slots
    n_frames: int
    admitted: bool = False
    finished: bool = False
    in_flight: bool = False
    next_frame: int = 0
    pending: collections.deque = dataclasses.field(default_factory=collections.deque)
    completed: int = 0


class Scheduler:
    """Admission by memory budget and continuous batch formation."""

    def __init__(self, budget_bytes, max_batch_items, max_batch_records, max_batch_cells, reserved_bytes=0):
        self.budget = int(budget_bytes)
        self.used = int(reserved_bytes)
        self.max_items = int(max_batch_items)
        self.max_records = int(max_batch_records)
        self.max_cells = int(max_batch_cells)
        self.sessions: dict[int, SessionState] = {}
        self.waiting: collections.deque = collections.deque()   # session ids not yet admitted
        self.log = []

    def add_session(self, sid, nbytes, samples, cells, n_frames):
        if samples > self.max_records or cells > self.max_cells:
            raise ValueError(f"session {sid} is larger than one launch")
        self.sessions[sid] = SessionState(sid, int(nbytes), int(samples), int(cells), int(n_frames))
        self.waiting.append(sid)

    def admit(self):
        """Admit waiting sessions in order while they fit the budget.
        Returns the newly admitted session ids."""
        out = []
        while self.waiting:
            s = self.sessions[self.waiting[0]]
            if self.used + s.bytes > self.budget:
                break
            self.waiting.popleft()
            self.used += s.bytes
            s.admitted = True
            out.append(s.sid)
        return out

    def arrive(self, req: Request):
        self.sessions[req.session].pending.append(req)

    def form_batch(self):
        """Oldest pending requests of admitted, idle sessions, within the
        per-launch item, record and cell capacity."""
        ready = [s for s in self.sessions.values() if s.admitted and not s.in_flight and s.pending]
        ready.sort(key=lambda s: s.pending[0].arrival)
        batch, recs, cells = [], 0, 0
        for s in ready:
            if len(batch) == self.max_items:
                break
            if recs + s.samples > self.max_records or cells + s.cells > self.max_cells:
                continue
            req = s.pending.popleft()
            s.in_flight = True
            batch.append(req)
            recs += s.samples
            cells += s.cells
        return batch

    def complete(self, batch, now):
        """Mark a launched batch done; returns the sessions that finished."""
        finished = []
        for req in batch:
            req.done = now
            s = self.sessions[req.session]
            s.in_flight = False
            s.completed += 1
            s.next_frame += 1
            self.log.append(req)
            if s.completed == s.n_frames:
                s.finished = True
                s.admitted = False
                self.used -= s.bytes
                finished.append(s.sid)
        return finished

    def idle(self):
        return all(s.finished for s in self.sessions.values())


def poisson_arrivals(rng, n, rate, start=0.0):
    """n arrival times of a Poisson process of the given rate (per second)."""
    return start + np.cumsum(rng.exponential(1.0 / rate, size=n))


def session_bytes(n_lights, n_points, table_size, cut_size, precision="fp32"):
    """Resident device bytes of one session: tree, grid, G-buffer, rgb."""
    n = n_lights
    tree = 64 * (2 * (n - 1)) + 64 * (2 * n - 1) + 64 * n + 4 * n + 8 * (n - 1) + 4 * (2 * n - 1) + 4 * n
    e = 4 if precision == "fp32" else 2
    grid = table_size * (8 + 8) + table_size * cut_size * (4 + 2 * e)
    return int(tree + grid + 40 * n_points)


class GpuExecutor:
    """Resident per-session device state and batched launches on two streams."""

    def __init__(self, torch, rll, device, max_items, max_records, max_cells, slots=2, keep_results=False,
                 timeline=False):
        self.torch, self.rll, self.dev = torch, rll, device
        self.keep_results = keep_results
        self.results = {}
        # (slot, start event, end event) of every launch, when asked for
        self.timeline = [] if timeline else None
        self.slots = []
        for _ in range(slots):
            stream = torch.cuda.Stream(device)
            ctx = rll.Context(device.index or 0, stream)
            batch = rll.Batch(ctx, max_items=max_items, max_records=max_records, max_cells=max_cells)
            self.slots.append(dict(stream=stream, ctx=ctx, batch=batch, busy=None, event=None))
        self.admin = rll.Context(device.index or 0, torch.cuda.current_stream(device))
        self.state = {}

    def reserved_bytes(self, max_records, max_cells):
        return len(self.slots) * (8 * max_records + 16 * max_records + 8 * max_cells)

    def create(self, sid, scene, precision="fp32", seed=None):
        torch, rll, dev = self.torch, self.rll, self.dev

        def T(a):
            return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

        d = dict(tri=T(scene.tris.reshape(-1, 9)), em=T(scene.emission), boxes=T(scene.boxes),
                 pos=T(scene.pos), nrm=T(scene.nrm), alb=T(scene.albedo))
        tree = rll.Tree(self.admin, d["tri"], d["em"])
        g = scene.grid
        grid = rll.Grid(self.admin, tree, rll.grid_params_for(g, precision=precision))
        del d["tri"], d["em"]
        rgb = torch.zeros(3, scene.n_points, device=dev)
        torch.cuda.synchronize(dev)
        self.state[sid] = dict(d=d, tree=tree, grid=grid, rgb=rgb, spp=scene.spp,
                               seed=scene.seed if seed is None else seed)

    def release(self, sid):
        st = self.state.pop(sid)
        if self.keep_results:
            self.torch.cuda.synchronize(self.dev)
            self.results[sid] = dict(rgb=st["rgb"].cpu().numpy(), grid=st["grid"].export())
        st["grid"].close()
        st["tree"].close()

    def free_slot(self):
        for i, sl in enumerate(self.slots):
            if sl["busy"] is None:
                return i
        return None

    def launch(self, slot, batch, frames):
        sl = self.slots[slot]
        items = []
        for req in batch:
            st = self.state[req.session]
            items.append(dict(grid=st["grid"], tree=st["tree"], pos=st["d"]["pos"], nrm=st["d"]["nrm"],
                              albedo=st["d"]["alb"], boxes=st["d"]["boxes"], seed=st["seed"],
                              frame=frames[req.session], spp=st["spp"], rgb=st["rgb"]))
        t0 = None
        if self.timeline is not None:
            t0 = self.torch.cuda.Event(enable_timing=True)
            t0.record(sl["stream"])
        sl["batch"].set_items(items)
        sl["batch"].run(do_split=True)
        ev = self.torch.cuda.Event(enable_timing=self.timeline is not None)
        ev.record(sl["stream"])
        if self.timeline is not None:
            self.timeline.append((slot, t0, ev))
        sl["busy"], sl["event"] = batch, ev

    def device_intervals(self):
        """(slot, start ms, end ms) of every launch on the device clock (CUDA
        events recorded on the slot's stream before its descriptor upload and
        after its pass), relative to the first launch's start."""
        self.torch.cuda.synchronize(self.dev)
        base = self.timeline[0][1]
        return [(slot, base.elapsed_time(a), base.elapsed_time(b)) for slot, a, b in self.timeline]

    def poll(self):
        """Slots whose batch has finished: list of (slot, batch)."""
        out = []
        for i, sl in enumerate(self.slots):
            if sl["busy"] is not None and sl["event"].query():
                out.append((i, sl["busy"]))
                sl["busy"], sl["event"] = None, None
        return out

    def status(self):
        return [sl["ctx"].sync_status() for sl in self.slots] + [self.admin.sync_status()]


def serve(executor, scheduler, scenes_by_sid, arrivals_by_sid, precision="fp32", clock=time.perf_counter,
          timeout_s=600.0):
    """Run the request loop until every session has finished. Returns the
    completed requests (with arrival / start / done times)."""
    events = sorted((t, sid, f) for sid, ts in arrivals_by_sid.items() for f, t in enumerate(ts))
    # sessions that fit at the start are opened before the first request
    for sid in scheduler.admit():
        executor.create(sid, scenes_by_sid[sid], precision)
    t0 = clock()
    k = 0
    while not scheduler.idle():
        now = clock() - t0
        if now > timeout_s:
            raise TimeoutError("serving loop did not finish")
        while k < len(events) and events[k][0] <= now:
            t, sid, f = events[k]
            scheduler.arrive(Request(sid, f, t))
            k += 1
        for sid in scheduler.admit():
            executor.create(sid, scenes_by_sid[sid], precision)
        for slot, batch in executor.poll():
            done = clock() - t0
            for sid in scheduler.complete(batch, done):
                executor.release(sid)
        slot = executor.free_slot()
        if slot is not None:
            batch = scheduler.form_batch()
            if batch:
                start = clock() - t0
                for r in batch:
                    r.start = start
                frames = {r.session: scheduler.sessions[r.session].next_frame for r in batch}
                executor.launch(slot, batch, frames)
                continue
        if k < len(events) or any(sl["busy"] is not None for sl in executor.slots):
            time.sleep(2e-5)
    return scheduler.log
