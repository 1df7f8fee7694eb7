"""Continuous batching of steady airfoil solves on one GPU.

A request is one steady solve (a solver configuration and its wall loops) with an arrival
time.  The service admits requests in arrival order while a solve slot is free and the
device-memory budget holds the new solve: the bytes a solve will allocate are known before
any allocation, from the host-only grid build of ``lbm_plan_geometry``.  An admitted solve
owns a CUDA stream and keeps all of its state on the device (populations, macroscopic
fields, wall records and its two captured step graphs) until it finishes.  Its level-0
steps are enqueued in chunks; after each chunk the host reads CL (eq 30) once and tests
convergence, comparing the mean CL over a window of chunks with the window before (the
window spans the acoustic round trip of the box, whose standing waves keep the sampled CL
oscillating long after the mean has settled).  Chunks of different solves run
concurrently on their streams: a multilevel solve of a few 1e4..1e5 cells per level fills a
fraction of the 152 SMs with each of its launches, so the solves in flight overlap on the
device.  Grid building (planning and ``lbm_set_geometry``) runs on worker threads while
the other solves keep the GPU busy; the step graphs are captured in thread-local mode, so
this does not disturb the streams of the running solves.

Each solve's arithmetic is the same whether it runs alone or in a mix: the kernels of one
solve read and write only that solve's buffers, and a solve's chunks run in stream order.
Only the FP64 atomic sums of the load integral may round differently between runs.

The backend is pluggable (``GpuBackend`` here; the CPU tests of the scheduling logic
drive a simulated one), so the admission, FIFO order and memory accounting are testable
without a GPU.
"""
from __future__ import annotations

import math
import os
import time
from collections import deque
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

__all__ = ["SolveRequest", "SolveResult", "Service", "GpuBackend", "summarize"]


@dataclass
class SolveRequest:
    rid: int
    arrival: float                  # seconds after the start of the run
    cfg: dict
    loops: list
    max_steps: int = 3000           # level-0 steps at most
    min_steps: int = 400            # no convergence test before this many level-0 steps
    check_every: int = 100          # level-0 steps per chunk (one CL read per chunk)
    window: int = 1                 # chunks per averaging window
    tol: float = 1e-3               # converged when the mean CL of the last window differs from
                                    # that of the window before by at most tol ...
    patience: int = 2               # ... on this many consecutive chunks


@dataclass
class SolveResult:
    rid: int
    status: str = "queued"          # converged | max_steps | diverged | rejected | error
    arrival: float = math.nan
    admitted: float = math.nan      # slot and memory granted, build starts
    started: float = math.nan       # first chunk enqueued
    finished: float = math.nan
    steps: int = 0
    CL: float = math.nan            # mean over the last window of chunk reads
    CD: float = math.nan
    device_bytes: float = 0.0
    node_updates_per_step: int = 0
    history: list = field(default_factory=list)   # (step, CL, CD) after each chunk
    message: str = ""

    @property
    def latency(self):
        """Time from arrival to the converged (or final) CL."""
        return self.finished - self.arrival


class _GpuHandle:
    def __init__(self, solver, stream, backend=None):
        import torch

        self.solver = solver
        self.stream = stream
        self.backend = backend
        self.event = torch.cuda.Event()

    def enqueue(self, n):
        self.solver.step_async(n)
        self.event.record(self.stream)

    def mark(self):
        """After a batched chunk: the chunk is done when this solve's stream reaches here."""
        self.event.record(self.stream)

    def ready(self):
        return self.event.query()

    def read(self):
        """Status check of the finished chunk, then CL/CD (raises LBMError on divergence)."""
        self.solver.synchronize()
        return self.solver.coefficients()

    def close(self):
        if self.backend is not None:
            self.backend.drop_batches(self)
        self.solver.close()


class GpuBackend:
    """Solves on the current CUDA device through the C ABI (one stream per solve, device
    memory from PyTorch's caching allocator through the allocation hooks).  step_batch
    advances several solves as lbm_batch batches (one launch per level-schedule node for
    all of them), regrouped whenever the set of solves changes."""

    def __init__(self):
        self._batches = {}           # group key -> [(member handles, Batch)]

    def step_batch(self, handles, n, key=0):
        """Advance the handles of one group by n level-0 steps as lbm_batch batches (one
        storage type per batch, at most 24 solves each), rebuilt when the group changes."""
        from . import Batch

        ids = [id(h) for h in handles]
        cur = self._batches.get(key, [])
        if [id(h) for grp, _ in cur for h in grp] != ids:
            self._drop(key)
            groups = {}
            for h in handles:
                groups.setdefault(h.solver.cfg.get("store", 0), []).append(h)
            cur = []
            for grp in groups.values():
                for i in range(0, len(grp), 24):
                    part = grp[i:i + 24]
                    cur.append((part, Batch([h.solver for h in part])))
            self._batches[key] = cur
            handles[:] = [h for grp, _ in cur for h in grp]
        for _, b in cur:
            b.step(n)
        for h in handles:
            h.mark()

    def _drop(self, key):
        for _, b in self._batches.pop(key, []):
            b.close()

    def drop_batches(self, handle=None):
        """Close the batches holding handle (every batch with handle None)."""
        for key in list(self._batches):
            if handle is None or any(handle is h for grp, _ in self._batches[key] for h in grp):
                self._drop(key)

    def plan(self, cfg, loops):
        from . import plan

        return plan(cfg, loops)

    def build(self, req):
        import torch

        from . import Solver

        stream = torch.cuda.Stream()
        s = Solver(req.cfg, stream=stream, torch_allocator=True)
        try:
            s.set_geometry(req.loops)
        except Exception:
            s.close()
            raise
        return _GpuHandle(s, stream, self)

    def free_bytes(self):
        import torch

        return torch.cuda.mem_get_info()[0]

    def host_threads(self, n):
        from . import set_host_threads

        set_host_threads(n)


class _Slot:
    __slots__ = ("req", "res", "handle", "need", "calm", "enqueued", "done", "released")

    def __init__(self, req, res, handle, need):
        self.req, self.res, self.handle, self.need = req, res, handle, need
        self.calm = 0
        self.enqueued = 0            # level-0 steps enqueued
        self.done = 0                # level-0 steps whose chunk has been read (batched mode)
        self.released = False


class Service:
    """Admission by slots and device-memory budget, FIFO; chunked stepping with CL checks.

    max_slots     solves resident at once (1 gives the one-solve-at-a-time baseline)
    mem_budget    device bytes the resident solves may hold (default: half the free memory)
    overhead      bytes added to each solve's plan (graphs, events, allocator rounding)
    builders      worker threads for planning and grid building; each build uses an equal
                  share of the host processors (concurrent builds that each took all of
                  them would oversubscribe the cores)
    batched       step the resident solves of the same level count together, in lockstep
                  chunks through the backend's step_batch (one launch per level-schedule node
                  for the group); groups advance independently, and a solve whose build
                  finishes during its group's chunk joins at the group's next chunk.  (One
                  lockstep group for all solves would hold the shallow solves to the pace
                  of the deepest one.)
    """

    def __init__(self, max_slots=8, mem_budget=None, overhead=16 << 20, builders=4, poll_s=2e-4, backend=None,
                 batched=False):
        self.batched = bool(batched)
        self.max_slots = int(max_slots)
        self.backend = backend or GpuBackend()
        self.mem_budget = mem_budget
        self.overhead = int(overhead)
        self.builders = int(builders)
        self.poll_s = poll_s
        self.trace = []              # (time, event, rid, resident bytes, resident solves)

    def run(self, requests, time_scale=1.0, on_finish=None, clock=None):
        """Serve the requests (arrivals scaled by time_scale); returns results by request order.
        on_finish(result, handle) runs before a finished solve releases its device memory."""
        clock = clock or time.perf_counter
        budget = self.mem_budget if self.mem_budget is not None else 0.5 * self.backend.free_bytes()
        results = {r.rid: SolveResult(rid=r.rid, arrival=r.arrival * time_scale) for r in requests}
        pending = deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        waiting = deque()            # (request, plan future), arrival order
        building = []                # (request, bytes, build future)
        active = []
        used = 0.0
        resident = 0                 # admitted and not yet finished
        self.trace = []
        t0 = clock()

        def now():
            return clock() - t0

        def note(ev, rid):
            self.trace.append((now(), ev, rid, used, resident))

        share = max(1, (os.cpu_count() or 1) // max(1, self.builders))
        set_threads = getattr(self.backend, "host_threads", None)

        def in_worker(fn, *args):
            if set_threads is not None:
                set_threads(share)
            return fn(*args)

        with ThreadPoolExecutor(max_workers=self.builders) as pool:
            try:
                while pending or waiting or building or active:
                    moved = False
                    t = now()
                    while pending and pending[0].arrival * time_scale <= t:
                        r = pending.popleft()
                        waiting.append((r, pool.submit(in_worker, self.backend.plan, r.cfg, r.loops)))
                        moved = True

                    # admission: arrival order; the head waits for memory (no overtaking)
                    while waiting and resident < self.max_slots:
                        r, pf = waiting[0]
                        if not pf.done():
                            break
                        res = results[r.rid]
                        try:
                            p = pf.result()
                        except Exception as e:   # geometry the grid builder rejects
                            waiting.popleft()
                            res.status, res.message, res.finished = "rejected", str(e), now()
                            moved = True
                            continue
                        need = float(p["device_bytes"]) + self.overhead
                        res.device_bytes = float(p["device_bytes"])
                        res.node_updates_per_step = int(p["node_updates_per_step"])
                        if need > budget:
                            waiting.popleft()
                            res.status, res.finished = "rejected", now()
                            res.message = f"needs {need:.3e} B, budget {budget:.3e} B"
                            moved = True
                            continue
                        if used + need > budget:
                            break
                        waiting.popleft()
                        used += need
                        resident += 1
                        res.admitted = now()
                        building.append((r, need, pool.submit(in_worker, self.backend.build, r)))
                        note("admit", r.rid)
                        moved = True

                    # finished builds start stepping
                    still = []
                    for r, need, bf in building:
                        if not bf.done():
                            still.append((r, need, bf))
                            continue
                        res = results[r.rid]
                        moved = True
                        try:
                            h = bf.result()
                        except Exception as e:
                            used -= need
                            resident -= 1
                            res.status, res.message, res.finished = "error", str(e), now()
                            note("error", r.rid)
                            continue
                        slot = _Slot(r, res, h, need)
                        res.started = now()
                        if self.batched:         # joins the next lockstep chunk
                            active.append(slot)
                            note("start", r.rid)
                            continue
                        try:
                            self._enqueue(slot)
                        except Exception as e:   # the solve could not be stepped: release it
                            h.close()
                            used -= need
                            resident -= 1
                            res.status, res.message, res.finished = "error", str(e), now()
                            note("error", r.rid)
                            continue
                        active.append(slot)
                        note("start", r.rid)
                    building = still

                    # batched: per level-count group, when the lockstep chunk of every member is
                    # done, every member reads CL; the continuing ones and the newcomers of the
                    # group step its next chunk together
                    if self.batched:
                        groups = {}
                        for slot in active:
                            groups.setdefault(self._group(slot), []).append(slot)
                        active = []
                        for key, grp in groups.items():
                            if not all(sl.handle.ready() for sl in grp if sl.enqueued > sl.done):
                                active += grp
                                continue
                            moved = True
                            keep = []
                            for slot in grp:
                                if slot.enqueued > slot.done:
                                    slot.done = slot.enqueued
                                    if not self._advance(slot, enqueue=False):
                                        self._finish(slot, now, on_finish, note)
                                        used -= slot.need
                                        resident -= 1
                                        continue
                                keep.append(slot)
                            if keep:
                                n = min(min(sl.req.check_every, sl.req.max_steps - sl.enqueued) for sl in keep)
                                handles = [sl.handle for sl in keep]
                                try:
                                    self.backend.step_batch(handles, n, key)
                                except Exception as e:
                                    for slot in keep:
                                        slot.res.status, slot.res.message = "error", str(e)
                                        self._finish(slot, now, on_finish, note)
                                        used -= slot.need
                                        resident -= 1
                                    keep = []
                                else:
                                    pos = {id(h): k for k, h in enumerate(handles)}
                                    keep.sort(key=lambda sl: pos[id(sl.handle)])
                                    for slot in keep:
                                        slot.enqueued += n
                            active += keep
                        if not moved:
                            time.sleep(self.poll_s)
                        continue

                    # chunks that completed: read CL, test convergence, continue or finish
                    keep = []
                    for slot in active:
                        if not slot.handle.ready():
                            keep.append(slot)
                            continue
                        moved = True
                        if self._advance(slot):
                            keep.append(slot)
                            continue
                        slot.res.finished = now()
                        try:
                            if on_finish is not None:
                                on_finish(slot.res, slot.handle)
                        finally:
                            slot.handle.close()
                            slot.released = True
                            used -= slot.need
                            resident -= 1
                            note("finish", slot.req.rid)
                    active = keep

                    if not moved:
                        time.sleep(self.poll_s)
            finally:
                # on an exception, release every solve still holding device memory
                for slot in active:
                    if not slot.released:
                        slot.handle.close()
                for _, _, bf in building:
                    try:
                        bf.result().close()
                    except Exception:
                        pass
        return [results[r.rid] for r in requests]

    @staticmethod
    def _group(slot):
        """Lockstep group of a solve in batched mode: its level count."""
        return slot.req.cfg.get("levels", 1)

    def _finish(self, slot, now, on_finish, note):
        slot.res.finished = now()
        try:
            if on_finish is not None:
                on_finish(slot.res, slot.handle)
        finally:
            slot.handle.close()
            slot.released = True
            note("finish", slot.req.rid)

    def _enqueue(self, slot):
        r = slot.req
        n = min(r.check_every, r.max_steps - slot.enqueued)
        slot.handle.enqueue(n)
        slot.enqueued += n

    def _advance(self, slot, enqueue=True):
        """Handle a completed chunk; True while the solve continues."""
        r, res = slot.req, slot.res
        try:
            c = slot.handle.read()
        except Exception as e:
            res.status, res.message, res.steps = "diverged", str(e), slot.enqueued
            return False
        res.steps = slot.enqueued
        res.history.append((slot.enqueued, c["CL"], c["CD"]))
        if not (math.isfinite(c["CL"]) and math.isfinite(c["CD"])):
            res.CL, res.CD = c["CL"], c["CD"]
            res.status = "diverged"
            return False
        w = max(1, r.window)
        last = res.history[-w:]
        res.CL = sum(h[1] for h in last) / len(last)
        res.CD = sum(h[2] for h in last) / len(last)
        if slot.enqueued >= r.min_steps and len(res.history) >= 2 * w:
            prev = sum(h[1] for h in res.history[-2 * w:-w]) / w
            slot.calm = slot.calm + 1 if abs(res.CL - prev) <= r.tol else 0
        else:
            slot.calm = 0
        if slot.calm >= r.patience:
            res.status = "converged"
            return False
        if slot.enqueued >= r.max_steps:
            res.status = "max_steps"
            return False
        if enqueue:
            self._enqueue(slot)
        return True


def summarize(results):
    """Latency percentiles (arrival to final CL), solves/hour over the makespan and counts."""
    done = [r for r in results if r.status in ("converged", "max_steps")]
    out = {k: sum(r.status == k for r in results) for k in ("converged", "max_steps", "diverged", "rejected", "error")}
    out["n"] = len(results)
    if not done:
        return out
    lat = np.array([r.latency for r in done])
    wait = np.array([r.admitted - r.arrival for r in done])
    t_first = min(r.arrival for r in results)
    t_last = max(r.finished for r in results if math.isfinite(r.finished))
    makespan = t_last - t_first
    updates = sum(r.node_updates_per_step * r.steps for r in done)
    out.update(p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
               mean_s=float(lat.mean()), wait_p50_s=float(np.percentile(wait, 50)),
               makespan_s=makespan, solves_per_hour=3600.0 * len(done) / makespan,
               node_updates=int(updates), glups=updates / makespan / 1e9)
    return out
