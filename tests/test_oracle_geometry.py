"""Pins of the oracle's grid builder (reading of the Sec 2.1 pre-processor: 2:1
distance bands, cell-centred solid test, cut links with the wall fraction q of
eq 27) against brute force with exact rational arithmetic on tiny grids, and of the
NACA input generator."""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from paper_2601_18443_gb300 import workloads as W

FIX = 4096


def snap(v, x0, hf):
    t = (v - x0) / hf * 4096.0
    return int(math.floor(t + 0.5)) if t >= 0 else -int(math.floor(-t + 0.5))


def segs_of(loops, cfg):
    hf = cfg["h0"] / 2 ** (cfg["levels"] - 1)
    out = []
    for lp in loops:
        pts = [(snap(x, cfg["x0"], hf), snap(y, cfg["y0"], hf)) for x, y in lp]
        out += [(pts[k], pts[(k + 1) % len(pts)]) for k in range(len(pts))]
    return out


def on_seg(a, b, p):
    cr = (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0])
    if cr != 0:
        return False
    t = (p[0] - a[0]) * (b[0] - a[0]) + (p[1] - a[1]) * (b[1] - a[1])
    return 0 <= t <= (b[0] - a[0]) ** 2 + (b[1] - a[1]) ** 2


def inside(segs, p):
    # vertical ray upwards (the oracle casts a horizontal one): independent even-odd count
    if any(on_seg(a, b, p) for a, b in segs):
        return True
    c = 0
    for a, b in segs:
        if (a[0] > p[0]) != (b[0] > p[0]):
            yc = Fr(a[1]) + Fr(p[0] - a[0]) * Fr(b[1] - a[1], b[0] - a[0])
            if yc > p[1]:
                c ^= 1
    return bool(c)


def dist2(a, b, p):
    dx, dy = b[0] - a[0], b[1] - a[1]
    t = Fr((p[0] - a[0]) * dx + (p[1] - a[1]) * dy, dx * dx + dy * dy)
    t = min(max(t, Fr(0)), Fr(1))
    qx, qy = a[0] + t * dx, a[1] + t * dy
    return (p[0] - qx) ** 2 + (p[1] - qy) ** 2


def centre(l, L, i, j):
    h = 2 ** (L - 1 - l) * FIX
    return ((2 * i + 1) * h // 2, (2 * j + 1) * h // 2)


CASES = {
    "arrow": (dict(levels=3, nx0=20, ny0=20, h0=1.0, layers=3),
              [np.array([[7.13, 8.02], [11.41, 9.37], [12.9, 6.23], [14.1, 10.6], [9.8, 13.31], [8.6, 10.9]])]),
    "two-bodies": (dict(levels=3, nx0=24, ny0=20, h0=0.5, x0=-1.0, y0=-2.0, layers=4),
                   [np.array([[2.03, 1.97], [4.2, 2.2], [3.1, 4.55]]), np.array([[6.3, 3.1], [8.0, 3.0], [8.1, 4.9], [6.2, 5.2]])]),
}


@pytest.mark.parametrize("name", list(CASES))
def test_level_masks_match_brute_force(name):
    over, loops = CASES[name]
    cfg = W.base_config(**over)
    s = oracle.Solver(cfg)
    s.set_geometry(loops)
    L = cfg["levels"]
    segs = segs_of(loops, cfg)
    # exact refinement radii: R_{L-1} = layers, R_l = R_{l+1} + layers 2^(L-1-l) (finest cells)
    R = [0] * L
    R[L - 1] = cfg["layers"] * FIX
    for l in range(L - 2, 0, -1):
        R[l] = R[l + 1] + cfg["layers"] * 2 ** (L - 1 - l) * FIX
    kind = {(i, j): "A" for i in range(cfg["nx0"]) for j in range(cfg["ny0"])}
    for l in range(L):
        if l > 0:
            prev = kind
            cov = {c for c, k in prev.items() if k == "A" and any(dist2(a, b, centre(l - 1, L, *c)) <= R[l] ** 2 for a, b in segs)}
            band = {c for c, k in prev.items() if k == "A" and c not in cov and any((c[0] + dx, c[1] + dy) in cov for dx in (-1, 0, 1) for dy in (-1, 0, 1))}
            kind = {}
            for (i, j) in cov | band:
                for a in (0, 1):
                    for b in (0, 1):
                        kind[(2 * i + a, 2 * j + b)] = "A" if (i, j) in cov else "G"
            covered_prev = cov
            # check the previous level now that its covered set is known
            check(s, l - 1, L, prev, covered_prev, segs)
    check(s, L - 1, L, kind, set(), segs)


def check(s, l, L, kind, covered, segs):
    F = s.get_fields(l)
    i0, j0, nx, ny = s.level_box(l)
    m = F["mask"]
    for (i, j), k in kind.items():
        sol = inside(segs, centre(l, L, i, j))
        exp = 5 if sol else (3 if (i, j) in covered else (4 if k == "G" else 1))
        got = int(m[j - j0, i - i0])
        if got == 2:
            got = 1
        assert got == exp, (l, i, j, got, exp)
    assert (m > 0).sum() == len(kind)


def test_cut_links_and_q_match_exact_intersections():
    over, loops = CASES["arrow"]
    cfg = W.base_config(**over)
    s = oracle.Solver(cfg)
    s.set_geometry(loops)
    L = cfg["levels"]
    segs = segs_of(loops, cfg)
    ijd, q = s.cut_links()
    CX = [0, 1, -1, 0, 0, 1, -1, 1, -1]
    CY = [0, 0, 0, 1, -1, 1, -1, -1, 1]
    F = s.get_fields(L - 1)
    i0, j0, nx, ny = s.level_box(L - 1)
    expected = set()
    for jj in range(ny):
        for ii in range(nx):
            if F["mask"][jj, ii] not in (1, 2):
                continue
            i, j = ii + i0, jj + j0
            for d in range(1, 9):
                if inside(segs, centre(L - 1, L, i - CX[d], j - CY[d])):
                    expected.add((i, j, d))
    assert {tuple(x) for x in ijd.tolist()} == expected
    for (i, j, d), qv in zip(ijd.tolist(), q):
        p = centre(L - 1, L, i, j)
        dv = (-CX[d] * FIX, -CY[d] * FIX)
        best = None
        for a, b in segs:
            ex, ey = b[0] - a[0], b[1] - a[1]
            den = dv[0] * ey - dv[1] * ex
            if den == 0:
                continue
            t = Fr((a[0] - p[0]) * ey - (a[1] - p[1]) * ex, den)
            u = Fr((a[0] - p[0]) * dv[1] - (a[1] - p[1]) * dv[0], den)
            if 0 <= t <= 1 and 0 <= u <= 1 and (best is None or t < best):
                best = t
        assert qv == pytest.approx(float(best), abs=1e-14)


def test_naca_generator():
    loop = W.naca_loop("0012", 1.0 / 256)
    x, y = loop[:, 0], loop[:, 1]
    n = len(loop)
    # symmetric section: the lower surface mirrors the upper one
    upper = loop[: (n + 2) // 2]
    lower = np.vstack([loop[:1], loop[(n + 2) // 2:][::-1], loop[n // 2:n // 2 + 1]])
    assert np.array_equal(upper[:, 0], lower[:, 0])
    assert np.array_equal(upper[:, 1], -lower[:, 1])
    # closed trailing edge, counter-clockwise, segments below h/2
    assert abs(y[0]) < 1e-12 and x[0] == pytest.approx(1.0)
    area = 0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y)
    assert area > 0
    # thickness integral: 10 t (0.2969*2/3 - 0.126/2 - 0.3516/3 + 0.2843/4 - 0.1036/5)
    assert area == pytest.approx(10 * 0.12 * (0.2969 * 2 / 3 - 0.063 - 0.3516 / 3 + 0.2843 / 4 - 0.1036 / 5), rel=1e-4)
    seg = np.linalg.norm(np.diff(np.vstack([loop, loop[:1]]), axis=0), axis=1)
    assert seg.max() <= 0.5 / 256 + 1e-15
    assert y.max() == pytest.approx(0.06, abs=2e-4)


def test_coincident_vertices_are_merged():
    # a wall polyline with repeated vertices describes the same wall: same grid, cut links and loads
    cfg = W.base_config(levels=2, nx0=48, ny0=32, h0=1.0, layers=4, Re=200.0, wall_model=3)
    base = np.array([[18.3, 12.2], [29.7, 13.1], [27.4, 19.6], [19.1, 18.4]])
    dup = np.array([base[0], base[1], base[1], base[2], base[3], base[3], base[3]])
    out = []
    for loop in (base, dup):
        s = oracle.Solver(cfg)
        s.set_geometry([loop])
        s.step(3)
        ld = s.get_loads()
        out.append(([s.get_fields(l)["mask"] for l in range(2)], s.cut_links(), ld))
    (ma, ca, la), (mb, cb, lb) = out
    assert all(np.array_equal(x, y) for x, y in zip(ma, mb))
    assert np.array_equal(ca[0], cb[0]) and np.array_equal(ca[1], cb[1])
    assert len(la["cp"]) == len(lb["cp"]) == 4
    for key in ("CL", "CD", "CDp", "CDf"):
        assert np.isfinite(lb[key]) and lb[key] == la[key]


def test_point_probes_agree_with_the_built_grid():
    # the probes serve sampled checks of grids too large to build; on a small grid they must
    # reproduce the full build: solid flags, refinement of level l+1 (covered cells), wall
    # distances and cut-link fractions
    cfg, loops = W.naca0012_small(levels=4)
    full = oracle.Solver(cfg)
    full.set_geometry(loops)
    probe = oracle.Solver(cfg)
    probe.set_walls(loops)
    for l in range(cfg["levels"]):
        F = full.get_fields(l)
        m = F["mask"]
        jj, ii = np.nonzero(m > 0)
        ij = np.stack([ii + F["i0"], jj + F["j0"]], axis=1)
        solid, near, dist = probe.probe_cells(l, ij)
        assert np.array_equal(solid.astype(bool), m[jj, ii] == 5)
        if l < cfg["levels"] - 1:
            # among the fluid cells that are not ghosts (which never refine), the covered ones
            # are exactly those within R_{l+1} of a wall
            sel = np.isin(m[jj, ii], (1, 2, 3))
            assert np.array_equal(near.astype(bool)[sel], m[jj, ii][sel] == 3)
        d = full.wall_distance(l)[jj, ii]
        fin = np.isfinite(d)
        assert np.array_equal(d[fin], dist[fin])
    ijd, q = full.cut_links()
    assert np.array_equal(probe.probe_links(ijd), q)
