"""Writes the golden grid summary of the NACA 0012 small workload.

The paper prints no worked example of the grid or of a time step, so the stored
values here are the oracle's own, written by this script (which calls only the
oracle and the shared input generators).  They guard the oracle's integer grid
build against accidental change; the paper-derived pins live in test_oracle_*.py.

Run:  python tests/golden/make_golden.py
"""
import hashlib
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2601_18443_gb300 import workloads as W  # noqa: E402


def summary():
    cfg, loops = W.naca0012_small()
    s = oracle.Solver(cfg)
    s.set_geometry(loops)
    lines = []
    for l in range(cfg["levels"]):
        F = s.get_fields(l)
        m = F["mask"]
        box = s.level_box(l)
        counts = [int((m == k).sum()) for k in range(6)]
        lines.append(f"level {l} box {box[0]} {box[1]} {box[2]} {box[3]} mask_counts " + " ".join(map(str, counts)))
    ijd, q = s.cut_links()
    h = hashlib.sha256(ijd.astype("<i4").tobytes()).hexdigest()[:16]
    lines.append(f"cut_links {len(ijd)} sha256_16 {h}")
    return lines


if __name__ == "__main__":
    with open(os.path.join(HERE, "naca0012_small_grid.txt"), "w") as f:
        f.write("# NACA 0012 small workload grid (oracle output, see make_golden.py)\n")
        f.write("\n".join(summary()) + "\n")
