"""lbm_autotune on the GPU: its choices are valid, and the tuned solve stays bit-identical
to an untuned one (every launch variant computes the same numbers), both through the
eager timing steps of all candidates and through the recaptured step graphs."""
import numpy as np
import pytest

import paper_2601_18443_gb300 as pkg
from paper_2601_18443_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("store", [0, 1])
def test_autotuned_solve_equals_the_default_one(store):
    pkg.build()
    cfg, loops = W.naca0012_small(levels=5)
    cfg = dict(cfg, store=store)
    a, b = pkg.Solver(cfg), pkg.Solver(cfg)
    a.set_geometry(loops)
    b.set_geometry(loops)
    a.step(3)
    b.step(3)                      # odd level-0 parity: the recapture starts from graph 1
    rep = b.autotune(steps=2)
    L = cfg["levels"]
    assert rep["steps_taken"] == 2 * 11 and rep["levels"] == L
    assert rep["candidates"] == [(m, st) for st in (0, 1) for m in (3, 4, 5, 6)]
    assert all(m in (3, 4, 5, 6) for m in rep["min_blocks"]) and rep["pdl"] in (0, 1)
    assert all(st in (0, 1) for st in rep["stage"])
    assert all(t > 0 for ts in rep["level_us"].values() for t in ts)
    assert rep["default_step_us"] > 0 and min(rep["step_us"].values()) > 0
    a.step(rep["steps_taken"])
    for l in range(L):
        assert np.array_equal(a.get_populations(l), b.get_populations(l), equal_nan=True), l
    a.step(25)
    b.step(25)
    for l in range(L):
        assert np.array_equal(a.get_populations(l), b.get_populations(l), equal_nan=True), l
    la, lb = a.coefficients(), b.coefficients()
    assert la["step"] == lb["step"] and abs(la["CL"] - lb["CL"]) < 1e-12
