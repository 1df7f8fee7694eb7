"""Launch timeline (lbm_set_timeline, lbm_get_timeline): one record per launch of each step
graph, in launch order, each launch past its wait only after the preceding one has ended
(programmatic dependent launch never lets a kernel's work overlap its predecessor's), and
the same populations as without the timeline."""
import numpy as np
import pytest

import paper_2601_18443_gb300 as pkg
from paper_2601_18443_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sched", [0, 1, 2, 3])
def test_timeline_orders_the_launches_and_leaves_the_solve_alone(sched):
    pkg.build()
    cfg, loops = W.naca0012_small(levels=5)
    L = cfg["levels"]
    a, b = pkg.Solver(cfg), pkg.Solver(cfg)
    for s in (a, b):
        s.set_geometry(loops)
        s.set_launch_variant([5] * L, 1, [sched] * L)
    assert b.timeline() == []
    b.set_timeline(True)
    a.step(6)
    b.step(6)
    tl = b.timeline()
    k = b.info()["kernels_per_step"]
    assert len(tl) == 2 * k
    for g in (0, 1):
        ev = [e for e in tl if e["graph"] == g]
        assert len(ev) == k
        # per graph: every level takes 2^l steps, and only levels with a finer one prolong
        steps = [e for e in ev if e["kind"] in (0, 1)]
        assert [sum(1 for e in steps if e["level"] == l) for l in range(L)] == [2 ** l for l in range(L)]
        assert all(e["level"] < L - 1 for e in ev if e["kind"] == 2)
        assert all(e["blocks"] > 0 and e["t_end_us"] > e["t_wait_us"] >= 0.0 for e in ev)
        assert min(e["t_wait_us"] for e in ev) == 0.0
        for p, q in zip(ev, ev[1:]):
            assert q["t_wait_us"] >= p["t_end_us"] - 0.05, (p, q)
    for l in range(L):
        x, y = a.get_populations(l), b.get_populations(l)
        assert np.array_equal(np.isnan(x), np.isnan(y)), l
        assert np.nanmax(np.abs(x - y)) <= 1e-6, l
    b.set_timeline(False)
    assert b.timeline() == []
    b.step(1)
