"""The level kernel's work lists, built on the host (no GPU): every tile and every 16 x 2-cell
warp that holds an active or ghost fluid cell appears exactly once, nothing else does, and
the lists run in non-increasing cost class (boundary-node work, then band or coalescing
cells, then other active cells, then ghost-only), recomputed here from the flag words."""
import numpy as np
import pytest

import paper_2601_18443_gb300 as pkg
from paper_2601_18443_gb300 import workloads as W

KIND_MASK, KIND_ACTIVE, KIND_GHOST = 0x3, 1, 3
FL_SOLID, FL_BAND, FL_BNODE = 1 << 2, 1 << 3, 1 << 4
COAL_MASK = 0xFF << 5


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()


def _cell_classes(fl, finest):
    """Per cell: -1 no work, 0 ghost fluid, 1 active fluid, 2 band or coalescing, 3 boundary node."""
    kind = fl & KIND_MASK
    fluid = (fl & FL_SOLID) == 0
    cls = np.full(fl.shape, -1, dtype=np.int64)
    cls[(kind == KIND_GHOST) & fluid] = 0
    act = (kind == KIND_ACTIVE) & fluid
    cls[act] = 1
    cls[act & ((fl & (FL_BAND | COAL_MASK)) != 0)] = 2
    if finest:
        cls[act & ((fl & FL_BNODE) != 0)] = 3
    return cls


def _expected(g, level, finest, warps):
    i0, j0, nx, ny = g.level_box(level)
    cls = _cell_classes(g.flags(level).reshape(ny, nx).astype(np.int64), finest)
    jj, ii = np.nonzero(cls >= 0)
    gi, gj = ii + i0, jj + j0
    if warps:
        lx, ly = gi & 31, gj & 7
        w = (lx >> 4) + 2 * (ly >> 1)
        keys = np.stack([gi - lx, gj - ly, w], axis=1)
    else:
        keys = np.stack([gi - (gi & 31), gj - (gj & 7), np.full(gi.shape, -1)], axis=1)
    out = {}
    for k, c in zip(map(tuple, keys), cls[jj, ii]):
        out[k] = max(out.get(k, -1), int(c))
    return out


def _case(name):
    if name == "naca0012-5lvl":
        return W.naca0012_small(levels=5)
    want = int(name.split("-")[1][0])
    for q in W.polar_requests(64):
        if q["levels"] == want:
            return W.polar_case(q)
    raise AssertionError(name)


@pytest.mark.parametrize("name", ["naca0012-5lvl", "polar-4lvl", "polar-5lvl"])
@pytest.mark.parametrize("warps", [False, True])
def test_work_lists_cover_the_work_once_in_cost_order(name, warps):
    cfg, loops = _case(name)
    g = pkg.Solver(cfg, host_only=True)
    g.set_geometry(loops)
    L = cfg["levels"]
    for l in range(L):
        want = _expected(g, l, l == L - 1, warps)
        got = [tuple(int(v) for v in r) for r in g.work_list(l, warps)]
        assert len(got) == len(set(got)), l                     # each entry once
        assert set(got) == set(want), l                         # exactly the entries with work
        classes = [want[k] for k in got]
        assert all(a >= b for a, b in zip(classes, classes[1:])), l
        if l == L - 1:
            assert classes[0] == 3                              # boundary-node work comes first
    g.close()


def _independent_levels(g, L):
    """Recomputed from the flag words: level l (1 <= l <= L - 2) is independent of the level
    above when no band cell has a ghost among its eight neighbours."""
    out = []
    for l in range(L):
        if not 1 <= l <= L - 2:
            out.append(False)
            continue
        i0, j0, nx, ny = g.level_box(l)
        fl = g.flags(l).reshape(ny, nx).astype(np.int64)
        ghost = np.pad((fl & KIND_MASK) == KIND_GHOST, 1)
        band = (fl & FL_BAND) != 0
        near = np.zeros((ny, nx), dtype=bool)
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                if di or dj:
                    near |= ghost[1 + dj:1 + dj + ny, 1 + di:1 + di + nx]
        out.append(not np.any(band & near))
    return out


def test_prolongation_grouping_follows_the_band_and_ghost_layout():
    # With exact distance bands a level's band cells lie `layers` of its cells inside its
    # ghost layer, so every level with a parent and a child is independent here, down to the
    # thinnest bands the wall-function stencil allows (6 layers); the host check guards the
    # grouping against layouts where that does not hold
    cases = [_case(n) for n in ("naca0012-5lvl", "polar-4lvl", "polar-5lvl")]
    cfg, loops = W.naca0012_small(levels=5)
    cases.append((dict(cfg, layers=6), loops))
    for cfg, loops in cases:
        g = pkg.Solver(cfg, host_only=True)
        g.set_geometry(loops)
        L = cfg["levels"]
        got = g.prolong_independence()
        assert got == _independent_levels(g, L)
        assert got == [False] + [True] * (L - 2) + [False]
        g.close()
