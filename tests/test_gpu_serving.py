"""The continuous-batching service on the GPU: each solve's result is the same alone and in a
mix of concurrently resident solves, the memory plan equals what a solve allocates, and
admission keeps the resident solves inside the memory budget."""
import numpy as np
import pytest

import paper_2601_18443_gb300 as pkg
from paper_2601_18443_gb300 import workloads as W
from paper_2601_18443_gb300.serve import GpuBackend, Service, SolveRequest, summarize

pytestmark = pytest.mark.gpu


def _requests(n=5, steps=300, levels=(4, 5), stagger=0.02):
    """n polar requests of the seeded stream with the given level counts; tol < 0 never
    converges, so every solve runs exactly `steps` level-0 steps."""
    out = []
    for q in W.polar_requests(64):
        if q["levels"] in levels:
            cfg, loops = W.polar_case(q)
            out.append(SolveRequest(rid=len(out), arrival=stagger * len(out), cfg=cfg, loops=loops,
                                    max_steps=steps, min_steps=0, check_every=100, tol=-1.0))
        if len(out) == n:
            break
    return out


def _serve(reqs, slots, budget=8 << 30, batched=False):
    snaps = {}

    def keep(res, h):
        s = h.solver
        L = s.cfg["levels"]
        snaps[res.rid] = (s.get_populations(0), s.get_populations(L - 1))

    svc = Service(max_slots=slots, mem_budget=budget, backend=GpuBackend(), batched=batched)
    res = svc.run(reqs, on_finish=keep)
    return svc, res, snaps


def test_plan_equals_the_allocation():
    pkg.build()
    req = _requests(1)[0]
    p = pkg.plan(req.cfg, req.loops)
    h = GpuBackend().build(req)
    try:
        info = h.solver.info()
        assert info["device_bytes"] == p["device_bytes"]
        assert info["cells_active"] == p["cells_active"]
        assert info["node_updates_per_step"] == p["node_updates_per_step"]
    finally:
        h.close()


def test_results_alone_equal_results_in_the_mix():
    pkg.build()
    reqs = _requests(5)
    _, alone, snaps_alone = _serve(reqs, slots=1)
    svc, mixed, snaps_mixed = _serve(reqs, slots=5)
    assert all(r.status == "max_steps" and r.steps == 300 for r in alone + mixed), \
        [(r.rid, r.status, r.steps, r.message) for r in alone + mixed]
    # the mix really overlapped: some solves were resident at the same time
    assert max(res for _, _, _, _, res in svc.trace) >= 2
    spans = sorted((r.started, r.finished) for r in mixed)
    assert any(spans[k + 1][0] < spans[k][1] for k in range(len(spans) - 1))
    for a, b in zip(alone, mixed):
        # populations bit for bit; CL/CD up to the order of the FP64 atomic sums of eq 30
        for pa, pb in zip(snaps_alone[a.rid], snaps_mixed[b.rid]):
            assert np.array_equal(pa, pb, equal_nan=True)
        ha, hb = np.array(a.history), np.array(b.history)
        assert ha.shape == hb.shape
        np.testing.assert_allclose(ha, hb, rtol=0, atol=1e-12)


def test_batched_service_results_equal_results_alone():
    # resident solves stepped together by batched launches (lbm_batch) give each solve's own
    # result: FP16 storage, so up to a few 16-bit units in the last place in the populations
    # and the 16-bit error level in the loads
    pkg.build()
    reqs = _requests(5, levels=(4, 5, 6))
    _, alone, snaps_alone = _serve(reqs, slots=1)
    svc, mixed, snaps_mixed = _serve(reqs, slots=5, batched=True)
    assert all(r.status == "max_steps" and r.steps == 300 for r in alone + mixed), \
        [(r.rid, r.status, r.steps, r.message) for r in alone + mixed]
    assert max(res for _, _, _, _, res in svc.trace) >= 2
    for a, b in zip(alone, mixed):
        for pa, pb in zip(snaps_alone[a.rid], snaps_mixed[b.rid]):
            assert np.array_equal(np.isnan(pa), np.isnan(pb))
            assert np.nanmax(np.abs(pa - pb)) <= 5e-4
        ha, hb = np.array(a.history), np.array(b.history)
        assert ha.shape == hb.shape and np.array_equal(ha[:, 0], hb[:, 0])
        scale = np.maximum(np.abs(ha[:, 1]), np.abs(ha[:, 2]))
        assert np.all(np.abs(ha[:, 1:] - hb[:, 1:]) <= 1e-2 * scale[:, None])


def test_memory_budget_limits_the_resident_solves():
    pkg.build()
    reqs = _requests(4, steps=200, stagger=0.0)
    plans = [pkg.plan(r.cfg, r.loops)["device_bytes"] for r in reqs]
    overhead = 16 << 20
    budget = sorted(plans)[-1] + sorted(plans)[-2] + 2 * overhead + 1   # two at a time at most
    svc = Service(max_slots=4, mem_budget=budget, overhead=overhead, backend=GpuBackend())
    res = svc.run(reqs)
    assert all(r.status == "max_steps" for r in res), [(r.rid, r.status, r.steps, r.message) for r in res]
    assert all(used <= budget for _, _, _, used, _ in svc.trace)
    assert max(n for _, _, _, _, n in svc.trace) <= 2
    s = summarize(res)
    assert s["max_steps"] == 4 and s["p50_s"] <= s["p99_s"]
