"""Device load history (lbm_set_load_history, lbm_get_load_history): records every N coarse
steps of what lbm_get_loads gives at those steps, the last `capacity` of them oldest first,
without changing the trajectory."""
import numpy as np
import pytest

import paper_2601_18443_gb300 as pkg
from paper_2601_18443_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_history_records_the_loads_of_the_sampled_steps():
    pkg.build()
    cfg, loops = W.naca0012_small(levels=4)
    L = cfg["levels"]
    a, b = pkg.Solver(cfg), pkg.Solver(cfg)
    a.set_geometry(loops)
    b.set_geometry(loops)
    assert b.load_history() == []
    b.set_load_history(every=5, capacity=8)
    want = {}
    for k in range(1, 48):
        a.step(1)
        if k % 5 == 0:
            want[k] = a.get_loads()
    b.step(7)
    b.step_async(40)
    h = b.load_history()
    assert [r["step"] for r in h] == list(range(10, 46, 5))          # 9 taken, the last 8 kept
    for r in h:
        w = want[r["step"]]
        for key in ("CL", "CD", "CDp", "CDf"):
            assert abs(r[key] - w[key]) <= 1e-12 * max(1.0, abs(w[key])), (r["step"], key)
        assert abs(r["mass"] - w["mass"]) <= 1e-12 * w["mass"]
    # the queries left the trajectory alone
    for l in range(L):
        assert np.array_equal(a.get_populations(l), b.get_populations(l), equal_nan=True), l
    b.set_load_history(every=0)
    b.step(10)
    assert b.load_history() == []
    with pytest.raises(pkg.LBMError):
        b.set_load_history(every=3, capacity=0)
