"""Host logic of the continuous-batching service, driven by a simulated backend (no GPU):
admission in arrival order under the slot and memory limits, rejection of solves that
cannot fit, convergence and divergence handling, memory release, and the summary."""
import math
import threading
import time

import pytest

from paper_2601_18443_gb300.serve import Service, SolveRequest, summarize


class FakeHandle:
    def __init__(self, be, req):
        self.be, self.req = be, req
        self.ready_at = 0.0
        self.steps = 0
        self.closed = False

    def enqueue(self, n):
        self.steps += n
        self.ready_at = time.perf_counter() + n * self.req.cfg["cost"]

    def ready(self):
        return time.perf_counter() >= self.ready_at

    def read(self):
        if self.req.cfg.get("diverge_at") and self.steps >= self.req.cfg["diverge_at"]:
            raise RuntimeError("lbm status -6: non-finite populations")
        if self.req.cfg.get("shedding"):     # periodic lift: never converges
            return dict(CL=0.5 + 0.1 * math.sin(self.steps / 70.0), CD=0.01)
        tau = self.req.cfg["tau"]
        cl = self.req.cfg["cl"] * (1.0 - math.exp(-self.steps / tau))
        return dict(CL=cl, CD=0.01)

    def close(self):
        assert not self.closed
        self.closed = True
        with self.be.lock:
            self.be.live -= 1


class FakeBackend:
    def __init__(self, free=1 << 30):
        self.free = free
        self.lock = threading.Lock()
        self.live = 0
        self.max_live = 0
        self.handles = []

    def plan(self, cfg, loops):
        if cfg.get("bad"):
            raise RuntimeError("lbm status -5: refinement reaches the level-0 box edge")
        return dict(device_bytes=cfg["bytes"], node_updates_per_step=cfg["updates"])

    def build(self, req):
        time.sleep(0.002)
        h = FakeHandle(self, req)
        with self.lock:
            self.live += 1
            self.max_live = max(self.max_live, self.live)
            self.handles.append(h)
        return h

    def free_bytes(self):
        return self.free


def make(rid, arrival, nbytes, cost=2e-5, tau=300.0, **kw):
    cfg = dict(bytes=nbytes, updates=1000 * (rid + 1), cost=cost, tau=tau, cl=0.5, **kw)
    return SolveRequest(rid=rid, arrival=arrival, cfg=cfg, loops=[], max_steps=4000, min_steps=200,
                        check_every=100, tol=2e-3, patience=2)


def check_trace(svc, budget, slots):
    for t, ev, rid, used, resident in svc.trace:
        assert used <= budget + 1e-6
        assert resident <= slots


def test_memory_budget_and_slots_are_never_exceeded():
    be = FakeBackend()
    reqs = [make(k, 0.001 * k, (3 + k % 4) << 20) for k in range(12)]
    budget = 16 << 20
    svc = Service(max_slots=3, mem_budget=budget, overhead=0, backend=be)
    res = svc.run(reqs)
    assert all(r.status == "converged" for r in res)
    check_trace(svc, budget, 3)
    assert be.max_live <= 3
    assert be.live == 0 and all(h.closed for h in be.handles)


def test_admission_follows_arrival_order():
    be = FakeBackend()
    # a large solve at the head holds back the small ones behind it until memory frees
    reqs = [make(0, 0.0, 6 << 20), make(1, 0.001, 9 << 20), make(2, 0.002, 1 << 20), make(3, 0.003, 1 << 20)]
    svc = Service(max_slots=4, mem_budget=10 << 20, overhead=0, backend=be)
    res = svc.run(reqs)
    order = [rid for _, ev, rid, _, _ in svc.trace if ev == "admit"]
    assert order == [0, 1, 2, 3]
    assert res[1].admitted >= res[0].finished
    assert all(r.status == "converged" for r in res)


def test_solves_that_cannot_fit_or_fail_to_plan_are_rejected():
    be = FakeBackend()
    reqs = [make(0, 0.0, 64 << 20), make(1, 0.0, 1 << 20, bad=True), make(2, 0.0, 1 << 20)]
    res = Service(max_slots=2, mem_budget=32 << 20, overhead=0, backend=be).run(reqs)
    assert [r.status for r in res] == ["rejected", "rejected", "converged"]
    assert "budget" in res[0].message and "box edge" in res[1].message


def test_divergence_ends_the_solve_and_frees_its_memory():
    be = FakeBackend()
    reqs = [make(0, 0.0, 4 << 20, diverge_at=300), make(1, 0.0, 4 << 20)]
    svc = Service(max_slots=1, mem_budget=8 << 20, overhead=0, backend=be)
    res = svc.run(reqs)
    assert res[0].status == "diverged" and res[0].steps == 300
    assert res[1].status == "converged"
    assert be.live == 0


def test_convergence_rule_and_step_cap():
    be = FakeBackend()
    fast, slow = make(0, 0.0, 1 << 20, tau=100.0), make(1, 0.0, 1 << 20, shedding=True)
    slow.max_steps = 500
    res = Service(max_slots=2, mem_budget=8 << 20, overhead=0, backend=be).run([fast, slow])
    # tau = 100: |dCL| over the chunk ending at n is 0.5 (e - 1) e^(-n/100), <= 2e-3 from n = 700;
    # two calm chunks in a row end the solve at n = 800
    assert res[0].status == "converged" and res[0].steps == 800
    assert [h[0] for h in res[0].history] == list(range(100, 900, 100))
    assert res[1].status == "max_steps" and res[1].steps == 500


def test_concurrent_slots_shorten_the_makespan_and_summary():
    reqs = [make(k, 0.0, 1 << 20, cost=5e-5) for k in range(6)]
    one = Service(max_slots=1, mem_budget=64 << 20, overhead=0, backend=FakeBackend()).run(reqs)
    many = Service(max_slots=6, mem_budget=64 << 20, overhead=0, backend=FakeBackend()).run(reqs)
    s1, s6 = summarize(one), summarize(many)
    assert s1["converged"] == s6["converged"] == 6
    assert s6["makespan_s"] < 0.6 * s1["makespan_s"]
    assert s6["p99_s"] < s1["p99_s"] and s6["solves_per_hour"] > s1["solves_per_hour"]
    assert s1["node_updates"] == sum(r.node_updates_per_step * r.steps for r in one)
    assert s1["p50_s"] <= s1["p99_s"]
    for a, b in zip(one, many):
        assert a.history == b.history


def test_window_mean_convergence_ignores_a_steady_oscillation():
    # CL = 0.8 + 0.05 sin(2 pi n / 400): chunk-to-chunk changes stay near 0.07, but the mean over
    # a 400-step window (4 chunks) is 0.8 exactly, so the windowed rule converges
    class Osc(FakeHandle):
        def read(self):
            return dict(CL=0.8 + 0.05 * math.sin(2 * math.pi * self.steps / 400.0), CD=0.01)

    class OscBackend(FakeBackend):
        def build(self, req):
            h = super().build(req)
            o = Osc(self, req)
            self.handles[-1] = o
            return o

    plain = make(0, 0.0, 1 << 20)
    plain.max_steps = 2000
    windowed = make(1, 0.0, 1 << 20)
    windowed.max_steps, windowed.window = 2000, 4
    be = OscBackend()
    res = Service(max_slots=2, mem_budget=8 << 20, overhead=0, backend=be).run([plain, windowed])
    assert res[0].status == "max_steps"
    assert res[1].status == "converged" and res[1].steps == 900
    assert res[1].CL == pytest.approx(0.8, abs=1e-12)


def test_a_solve_that_cannot_be_stepped_is_released():
    class Broken(FakeHandle):
        def enqueue(self, n):
            raise RuntimeError("lbm status -3: launch failed")

    class BrokenBackend(FakeBackend):
        def build(self, req):
            h = super().build(req)
            if req.cfg.get("broken"):
                b = Broken(self, req)
                self.handles[-1] = b
                return b
            return h

    be = BrokenBackend()
    reqs = [make(0, 0.0, 4 << 20, broken=True), make(1, 0.0, 4 << 20)]
    svc = Service(max_slots=1, mem_budget=8 << 20, overhead=0, backend=be)
    res = svc.run(reqs)
    assert res[0].status == "error" and "launch failed" in res[0].message
    assert res[1].status == "converged"
    assert be.live == 0 and all(h.closed for h in be.handles)


def test_an_exception_in_the_caller_hook_still_releases_every_solve():
    be = FakeBackend()
    reqs = [make(k, 0.0, 1 << 20, cost=1e-5 * (k + 1)) for k in range(4)]

    def boom(res, handle):
        raise ValueError("caller hook failed")

    with pytest.raises(ValueError):
        Service(max_slots=4, mem_budget=64 << 20, overhead=0, backend=be).run(reqs, on_finish=boom)
    time.sleep(0.05)
    assert be.live == 0


def test_builders_share_the_host_processors():
    # every plan and build runs on a worker thread that first limits its grid-build threads
    # to an equal share of the processors
    import os

    class Recording(FakeBackend):
        def __init__(self):
            super().__init__()
            self.calls = []

        def host_threads(self, n):
            with self.lock:
                self.calls.append((threading.get_ident(), n))

    be = Recording()
    reqs = [make(k, 0.0, 1 << 20) for k in range(6)]
    res = Service(max_slots=3, mem_budget=1 << 30, builders=3, backend=be).run(reqs)
    assert all(r.status == "converged" for r in res)
    share = max(1, (os.cpu_count() or 1) // 3)
    assert len(be.calls) == 12 and all(n == share for _, n in be.calls)
    assert threading.get_ident() not in {t for t, _ in be.calls}


def test_host_thread_count_leaves_the_grid_unchanged():
    import paper_2601_18443_gb300 as pkg
    from paper_2601_18443_gb300 import workloads as W
    pkg.build()
    cfg, loops = W.naca0012_small(levels=4)
    ref = pkg.grid_digest(cfg, loops)
    try:
        pkg.set_host_threads(1)
        assert pkg.grid_digest(cfg, loops) == ref
        pkg.set_host_threads(3)
        assert pkg.grid_digest(cfg, loops) == ref
    finally:
        pkg.set_host_threads(0)


class BatchingBackend(FakeBackend):
    """Steps all handles of a batch together (the cost of the batch's slowest member) and
    records the chunks it was given."""

    def __init__(self, **kw):
        super().__init__(**kw)
        self.chunks = []               # (member rids, steps)

    def step_batch(self, handles, n, key=0):
        self.chunks.append(([h.req.rid for h in handles], n, key))
        cost = max(h.req.cfg["cost"] for h in handles)
        t = time.perf_counter() + n * cost
        for h in handles:
            h.steps += n
            h.ready_at = t


def test_batched_mode_steps_members_in_lockstep_with_the_same_results():
    reqs = [make(k, 0.002 * k, 1 << 20, cost=2e-5, tau=100.0 + 30 * k) for k in range(6)]
    reqs[4].cfg["diverge_at"] = 400
    for k, r in enumerate(reqs):
        r.cfg["levels"] = 4 + k % 2          # two lockstep groups
    be = BatchingBackend()
    svc = Service(max_slots=3, mem_budget=64 << 20, overhead=0, backend=be, batched=True)
    res = svc.run(reqs)
    alone = Service(max_slots=3, mem_budget=64 << 20, overhead=0, backend=FakeBackend()).run(reqs)
    # same statuses, step counts and CL histories as the unbatched service
    for a, b in zip(alone, res):
        assert (a.status, a.steps) == (b.status, b.steps)
        assert a.history == b.history
    assert res[4].status == "diverged" and res[4].steps == 400
    # every chunk steps each member by the same count; no chunk holds more than the slots;
    # a chunk holds solves of one level count only
    assert all(n == 100 for _, n, _ in be.chunks)
    assert all(len(m) <= 3 for m, _, _ in be.chunks)
    assert all({reqs[rid].cfg["levels"] for rid in m} == {key} for m, _, key in be.chunks)
    # a member appears in consecutive chunks of its group from its first to its last
    for r in res:
        key = reqs[r.rid].cfg["levels"]
        mine = [m for m, _, k in be.chunks if k == key]
        seen = [k for k, m in enumerate(mine) if r.rid in m]
        assert seen == list(range(seen[0], seen[-1] + 1))
        assert len(seen) * 100 == r.steps
    check_trace(svc, 64 << 20, 3)
    assert be.live == 0 and all(h.closed for h in be.handles)
