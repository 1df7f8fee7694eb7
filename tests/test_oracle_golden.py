"""Regression guard of the oracle's integer grid build (values written by
tests/golden/make_golden.py from the oracle itself)."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def test_grid_summary_unchanged():
    with open(os.path.join(HERE, "golden", "naca0012_small_grid.txt")) as f:
        stored = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    assert make_golden.summary() == stored
