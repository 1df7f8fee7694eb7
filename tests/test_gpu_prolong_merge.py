"""Grouped prolongation launches (lbm_set_prolong_merge): a solve whose prolongations of
consecutive levels share launches computes what the solve with one launch per prolongation
computes, up to FP32 rounding (the grouped launch runs the same per-cell code in the batched
kernel's instantiation), and issues fewer kernels per coarse step."""
import numpy as np
import pytest

import paper_2601_18443_gb300 as pkg
from paper_2601_18443_gb300 import workloads as W

pytestmark = pytest.mark.gpu

POP_TOL = 1e-6


def _case(name):
    if name == "naca0012-5lvl":
        return W.naca0012_small(levels=5)
    for q in W.polar_requests(256):
        if q["levels"] == 6:
            return W.polar_case(q)
    raise AssertionError("no 6-level request")


@pytest.mark.parametrize("name", ["naca0012-5lvl", "polar-6lvl"])
def test_grouped_prolongations_compute_the_same_numbers(name):
    pkg.build()
    cfg, loops = _case(name)
    L = cfg["levels"]
    a, b = pkg.Solver(cfg), pkg.Solver(cfg)
    a.set_geometry(loops)
    b.set_geometry(loops)
    n_a = a.set_prolong_merge(False)
    n_b = b.set_prolong_merge(True)
    assert n_a == n_b and 0 <= n_b <= L - 2
    ka, kb = a.info()["kernels_per_step"], b.info()["kernels_per_step"]
    if n_b > 0:
        assert kb < ka
    else:
        assert kb == ka
    a.step(3)
    b.step(3)
    a.step(40)
    b.step(40)
    for l in range(L):
        x, y = a.get_populations(l), b.get_populations(l)
        assert np.array_equal(np.isnan(x), np.isnan(y)), l
        assert np.nanmax(np.abs(x - y)) <= POP_TOL, l
    la, lb = a.get_loads(), b.get_loads()
    assert la["step"] == lb["step"] == 43
    assert abs(la["mass"] - lb["mass"]) <= 1e-7 * la["mass"]
