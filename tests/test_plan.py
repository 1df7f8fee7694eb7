"""lbm_plan_geometry runs the host grid build without a GPU: its active-cell counts
equal the oracle's, and its memory plan grows with the grid."""
import numpy as np
import pytest

import oracle
import paper_2601_18443_gb300 as pkg
from paper_2601_18443_gb300 import workloads as W


def test_plan_counts_match_the_oracle():
    pkg.build()
    cfg, loops = __import__("__graft_entry__").smoke_case()
    p = pkg.plan(cfg, loops)
    r = oracle.Solver(cfg)
    r.set_geometry(loops)
    for l in range(cfg["levels"]):
        m = r.get_fields(l)["mask"]
        assert p["cells_active"][l] == int(((m == 1) | (m == 2)).sum())
    assert p["node_updates_per_step"] == sum(n << l for l, n in enumerate(p["cells_active"]))
    assert p["wall_records"] == len(r.wall_records()[0])
    assert p["device_bytes"] > 0


def test_plan_memory_grows_with_the_grid_and_the_storage():
    pkg.build()
    small = pkg.plan(*W.naca0012_small(levels=4))
    big = pkg.plan(*W.naca0012_small(levels=6))
    assert big["device_bytes"] > small["device_bytes"]
    cfg, loops = W.naca0012_small(levels=6)
    half = pkg.plan(dict(cfg, store=1), loops)
    assert half["device_bytes"] < big["device_bytes"]


def test_plan_reports_geometry_errors():
    pkg.build()
    cfg = W.base_config(levels=3, nx0=32, ny0=32, h0=1.0, layers=3)
    with pytest.raises(pkg.LBMError) as e:
        pkg.plan(cfg, [W.rectangle(0.5, 0.5, 5.0, 5.0)])     # refinement reaches the box edge
    assert e.value.code == -5 and "box edge" in str(e.value)


def test_plan_rejects_degenerate_loops():
    pkg.build()
    cfg = W.base_config(levels=2, nx0=64, ny0=64, h0=1.0, layers=4)
    with pytest.raises(pkg.LBMError) as e:
        pkg.plan(cfg, [np.array([[20.0, 20.0], [30.0, 30.0]])])          # two vertices
    assert e.value.code == -5 and "3 vertices" in str(e.value)
    with pytest.raises(pkg.LBMError) as e:
        pkg.plan(cfg, [np.array([[20.0, 20.0], [30.0, 30.0], [40.0, 40.0]])])   # zero area
    assert e.value.code == -5 and "degenerate" in str(e.value)


def test_plan_rejects_crossing_loops_and_accepts_touching_ones():
    pkg.build()
    cfg = W.base_config(levels=2, nx0=64, ny0=64, h0=1.0, layers=4)
    # two overlapping squares: their edges cross
    with pytest.raises(pkg.LBMError) as e:
        pkg.plan(cfg, [W.rectangle(20.0, 20.0, 30.0, 30.0), W.rectangle(25.0, 25.0, 35.0, 35.0)])
    assert e.value.code == -5 and "cross" in str(e.value)
    # a figure eight with lobes of different size (nonzero signed area, one self-crossing)
    eight = np.array([[20.0, 20.0], [36.0, 32.0], [36.0, 20.0], [20.0, 28.0]])
    with pytest.raises(pkg.LBMError) as e:
        pkg.plan(cfg, [eight])
    assert e.value.code == -5 and "cross" in str(e.value)
    # loops that only touch along an edge, and separate loops, are valid geometry
    pkg.plan(cfg, [W.rectangle(20.0, 20.0, 30.0, 30.0), W.rectangle(30.0, 22.0, 38.0, 28.0)])
    pkg.plan(cfg, [W.rectangle(18.0, 18.0, 26.0, 26.0), W.rectangle(32.0, 32.0, 42.0, 42.0)])


_DIGEST_SCRIPT = r"""
import sys
import paper_2601_18443_gb300 as pkg
from paper_2601_18443_gb300 import workloads as W
cases = [W.naca0012_small(levels=6), W.highlift_3element(levels=4, layers=16, box=(4.0, 2.0), h0=1.0 / 64.0)]
cases += [W.polar_case(r) for r in W.polar_requests(3)]
cases.append((W.base_config(levels=2, nx0=64, ny0=64, h0=1.0, layers=4),
              [W.rectangle(10, 10, 15, 15), W.rectangle(30.0, 30.0, 44.0, 38.0)]))
print(" ".join(str(pkg.grid_digest(c, l)) for c, l in cases))
# rejected inputs: the same message whatever the thread count (the first violation in scan order)
bad = [(W.base_config(levels=3, nx0=32, ny0=32, h0=1.0, layers=3), [W.rectangle(0.5, 0.5, 5.0, 5.0)]),
       (W.base_config(levels=3, nx0=64, ny0=64, h0=1.0, layers=1), [W.rectangle(28, 28, 36, 36)]),
       (W.base_config(levels=2, nx0=64, ny0=64, h0=1.0, layers=4),
        [W.rectangle(20.0, 20.0, 30.0, 30.0), W.rectangle(25.0, 25.0, 35.0, 35.0)])]
for c, l in bad:
    try:
        pkg.plan(c, l)
        print("accepted")
    except pkg.LBMError as e:
        print(str(e))
"""


def test_grid_build_does_not_depend_on_the_host_thread_count():
    # the builder's parallel passes (table fill, nesting checks, cut links, wall records,
    # tiles, wall distance) must give the same tables byte for byte with 1, 3 or 8 threads
    import os
    import subprocess
    import sys
    pkg.build()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for nt in ("1", "3", "8"):
        env = dict(os.environ, OMP_NUM_THREADS=nt, PYTHONPATH=root)
        r = subprocess.run([sys.executable, "-c", _DIGEST_SCRIPT], capture_output=True, text=True, env=env,
                           cwd=root, timeout=300)
        assert r.returncode == 0, r.stderr
        outs.append(r.stdout.splitlines())
    digests = outs[0][0].split()
    assert len(digests) == 6 and all(int(d) != 0 for d in digests)
    assert len(outs[0]) == 4 and all("accepted" not in m for m in outs[0][1:])
    assert outs[0] == outs[1] == outs[2]
    # the digest sees a change of the input
    cfg, loops = W.naca0012_small(levels=3)
    assert pkg.grid_digest(cfg, loops) != pkg.grid_digest(cfg, [loops[0] + 1e-3])


def test_grid_digest_reports_geometry_errors():
    pkg.build()
    cfg = W.base_config(levels=2, nx0=64, ny0=64, h0=1.0, layers=4)
    with pytest.raises(pkg.LBMError) as e:
        pkg.grid_digest(cfg, [W.rectangle(20.0, 20.0, 30.0, 30.0), W.rectangle(25.0, 25.0, 35.0, 35.0)])
    assert e.value.code == -5
