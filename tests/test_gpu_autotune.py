"""lbm_autotune on the GPU: its choices are valid, and the tuned solve stays bit-identical
to an untuned one (every launch variant computes the same numbers), both through the
eager timing steps of all candidates and through the recaptured step graphs; and each
variant set directly gives the same populations as the default."""
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
    assert rep["steps_taken"] == 2 * 10 and rep["levels"] == L
    assert min(rep["step_us_confirm"].values()) > 0
    assert rep["candidates"] == [(5, 0), (6, 0), (5, 1), (6, 1)]
    assert all(pe in (0, 1) for pe in rep["persistent"])
    assert all(m in (5, 6) for m in rep["min_blocks"]) and rep["pdl"] in (0, 1)
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


@pytest.mark.parametrize("mb,pdl,pe", [(6, 1, 0), (5, 0, 0), (6, 0, 1), (5, 1, 1), (6, 1, 1)])
def test_each_launch_variant_computes_the_same_numbers(mb, pdl, pe):
    pkg.build()
    cfg, loops = W.naca0012_small(levels=5)
    L = cfg["levels"]
    a, b = pkg.Solver(cfg), pkg.Solver(cfg)
    a.set_geometry(loops)
    b.set_geometry(loops)
    b.set_launch_variant([mb] * L, pdl, [pe] * L)
    a.step(6)
    b.step(6)
    for l in range(L):
        assert np.array_equal(a.get_populations(l), b.get_populations(l), equal_nan=True), l
    with pytest.raises(pkg.LBMError):
        b.set_launch_variant([4] * L, 1)
    # queries in between leave the trajectory alone
    a.coefficients(); b.coefficients()
    a.step(3); b.step(3)
    for l in range(L):
        assert np.array_equal(a.get_populations(l), b.get_populations(l), equal_nan=True), l
