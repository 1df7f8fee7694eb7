"""Parity of the product's host grid builder with the oracle's, without a GPU.

A host-only handle (lbm_create_host) builds the same tables lbm_set_geometry uploads
to the device.  Integer tables (level boxes, cell masks, cut-link sets, wall-record
stencils) and the FP64 geometry the builder derives (wall distances, wall fractions q of
eq 27, wall-point geometry of Sec 2.3) must equal the oracle's bit for bit: both evaluate
the same exact predicates on the same snapped vertices (Sec 2.1 pre-processor reading)."""
import numpy as np
import pytest

import oracle
import paper_2601_18443_gb300 as pkg
from paper_2601_18443_gb300 import workloads as W


def _polar(k):
    return lambda: W.polar_case(W.polar_requests(12)[k])


CASES = {
    "naca2412-3lvl": lambda: __import__("__graft_entry__").smoke_case(),
    "naca0012-6lvl": lambda: W.naca0012_small(),
    "three-element-4lvl": lambda: W.highlift_3element(levels=4, layers=16, box=(4.0, 2.0), h0=1.0 / 64.0),
    # seeded polar requests: cambered sections at several angles and 5 or 6 levels
    "polar-3313-a1.6-5lvl": _polar(1),
    "polar-4409-a9.3-5lvl": _polar(2),
    "polar-3414-a14-5lvl": _polar(6),
    "polar-3418-a-4-5lvl": _polar(11),
    "polar-4514-a2.9-6lvl": _polar(5),
    "square-L-diamond-3lvl": lambda: (W.base_config(levels=3, nx0=96, ny0=64, h0=1.0, layers=3),
                                      [W.rectangle(12, 12, 20, 20), W.l_shape(40, 20, 56, 36, 48, 28),
                                       np.array([[78.0, 20.0], [86.0, 28.0], [78.0, 36.0], [70.0, 28.0]])]),
    "touching-rectangles-2lvl": lambda: (W.base_config(levels=2, nx0=64, ny0=64, h0=1.0, layers=4),
                                         [W.rectangle(20.0, 20.0, 30.0, 30.0), W.rectangle(30.0, 22.0, 38.0, 28.0)]),
    "two-loops-periodic-3lvl": lambda: (
        W.base_config(levels=3, nx0=64, ny0=64, h0=1.0, layers=3, periodic=1, solid_walls=0),
        [W.rectangle(10, 10, 15, 15), np.array([[40.0, 30.0], [50.0, 40.0], [40.0, 50.0], [30.0, 40.0]])]),
    "sliver-triangle-2lvl": lambda: (
        W.base_config(levels=2, nx0=32, ny0=32, h0=1.0, layers=4, wall_model=2),
        [np.array([[8.0, 16.505], [24.0, 16.503], [24.0, 16.507]])]),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    oracle.build()


@pytest.mark.parametrize("name", list(CASES))
def test_host_grid_tables_equal_the_oracle(name):
    cfg, loops = CASES[name]()
    g = pkg.Solver(cfg, host_only=True)
    g.set_geometry(loops)
    r = oracle.Solver(cfg)
    r.set_geometry(loops)
    for l in range(cfg["levels"]):
        assert g.level_box(l) == r.level_box(l), f"level {l}"
        assert np.array_equal(g.mask(l), r.get_fields(l)["mask"]), f"level {l}"
        dg, dr = g.wall_distance(l), r.wall_distance(l)
        assert np.array_equal(np.isfinite(dg), np.isfinite(dr)), f"level {l}"
        fin = np.isfinite(dr)
        assert np.array_equal(dg[fin], dr[fin]), f"level {l}"
    for a, b in zip(g.cut_links(), r.cut_links()):
        assert np.array_equal(a, b)
    for a, b in zip(g.wall_records(), r.wall_records()):
        assert np.array_equal(a, b)
    g.close()


def test_host_only_handle_refuses_device_work():
    cfg, loops = __import__("__graft_entry__").smoke_case()
    g = pkg.Solver(cfg, host_only=True)
    with pytest.raises(pkg.LBMError) as e:
        g.level_box(0)
    assert e.value.code == -4
    g.set_geometry(loops)
    for call in (lambda: g.step(1), lambda: g.get_fields(0), lambda: g.get_loads(), lambda: g.get_state(),
                 lambda: g.get_populations(0), lambda: g.wall_state(), lambda: g.info(), lambda: g.autotune(1),
                 lambda: g.set_timeline(True), lambda: g.set_load_history(5, 8),
                 lambda: g.set_prolong_merge(False), lambda: g.set_launch_variant([5] * 6, 1, [3] * 6)):
        with pytest.raises(pkg.LBMError) as e:
            call()
        assert e.value.code == -4
    assert g.mask(0).shape == g.level_box(0)[:1:-1]
    g.close()
    g.close()


@pytest.mark.parametrize("name", ["naca0012-6lvl", "three-element-4lvl", "polar-3414-a14-5lvl"])
def test_reference_point_stencils_and_weights(name):
    # step 1 of Sec 2.3 as the device applies it: the stencil is the 4 x 4 block of finest
    # cells around R without solid cells and boundary nodes (reading of the unspecified
    # stencil); rho_R uses normalised inverse-squared-distance weights; u_R the intercept of
    # the linear least-squares fit, recomputed here with numpy's pseudo-inverse
    cfg, loops = CASES[name]()
    g = pkg.Solver(cfg, host_only=True)
    g.set_geometry(loops)
    L = cfg["levels"]
    i0, j0, nx, ny = g.level_box(L - 1)
    mask = g.mask(L - 1)
    sij, wr, wu = g.wall_stencils()
    ij, geo, ns = g.wall_records()
    assert len(sij) == len(ij) > 0
    for r in range(len(ij)):
        rx, ry = geo[r, 5], geo[r, 6]
        ic, jc = int(np.floor(rx - 0.5)), int(np.floor(ry - 0.5))
        want = [(ic + a, jc + b) for b in range(-1, 3) for a in range(-1, 3)
                if mask[jc + b - j0, ic + a - i0] == 1]
        n = ns[r]
        got = [tuple(x) for x in sij[r, :n]]
        assert got == want, r
        assert np.all(sij[r, n:] == -1) and np.all(wr[r, n:] == 0) and np.all(wu[r, n:] == 0)
        dx = np.array([i + 0.5 - rx for i, _ in got])
        dy = np.array([j + 0.5 - ry for _, j in got])
        inv = 1.0 / (dx * dx + dy * dy)
        np.testing.assert_allclose(wr[r, :n], inv / inv.sum(), rtol=1e-12, atol=0)
        phi = np.stack([np.ones(n), dx, dy], axis=1)
        np.testing.assert_allclose(wu[r, :n], np.linalg.pinv(phi)[0], rtol=0, atol=1e-12)
        # the intercept row reproduces any linear field at R
        a, b, c = 0.7, -1.3, 2.1
        assert abs(wu[r, :n] @ (a + b * dx + c * dy) - a) < 1e-12
    g.close()


@pytest.mark.parametrize("name", ["naca2412-3lvl", "three-element-4lvl", "square-L-diamond-3lvl"])
def test_surface_elements_take_the_two_nearest_boundary_nodes(name):
    # Sec 3.1.3 reading: each surface segment takes C_p, C_f from the two boundary nodes
    # nearest to its midpoint (ties to the lower record index), weighted by 1/d^2;
    # brute force over all records here
    cfg, loops = CASES[name]()
    g = pkg.Solver(cfg, host_only=True)
    g.set_geometry(loops)
    mid, b12, w12 = g.segment_map()
    ij, _, _ = g.wall_records()
    centres = ij.astype(np.float64) + 0.5
    assert len(mid) > 0 and len(ij) >= 2
    for k in range(len(mid)):
        d2 = ((centres - mid[k]) ** 2).sum(axis=1)
        order = np.lexsort((np.arange(len(d2)), d2))
        assert tuple(b12[k]) == (order[0], order[1]), k
        np.testing.assert_allclose(w12[k], 1.0 / d2[order[:2]], rtol=1e-12)
    g.close()


def test_host_only_handle_argument_checks():
    import ctypes as C
    lib = pkg.library()
    cfg, loops = __import__("__graft_entry__").smoke_case()
    # invalid configurations are refused before any work
    bad = pkg._config_struct(dict(cfg, levels=0))
    h = C.c_void_p()
    assert lib.lbm_create_host(C.byref(bad), C.byref(h)) == -1 and not h.value
    assert lib.lbm_create_host(None, C.byref(h)) == -1
    g = pkg.Solver(cfg, host_only=True)
    g.set_geometry(loops)
    # capacities below the level box are refused; a level out of range too
    i0, j0, nx, ny = g.level_box(0)
    d = np.zeros(nx * ny - 1)
    assert lib.lbm_get_wall_distance(g._h, 0, pkg._dp(d), nx * ny - 1) == -1
    with pytest.raises(pkg.LBMError):
        g.level_box(cfg["levels"])
    # a second geometry replaces the first; a rejected one leaves no tables behind
    before = g.mask(cfg["levels"] - 1).copy()
    g.set_geometry(loops)
    assert np.array_equal(g.mask(cfg["levels"] - 1), before)
    with pytest.raises(pkg.LBMError):
        g.set_geometry([np.array([[0.0, 0.0], [1.0, 1.0]])])
    with pytest.raises(pkg.LBMError) as e:
        g.level_box(0)
    assert e.value.code == -4
    g.close()


CX = [0, 1, -1, 0, 0, 1, -1, 1, -1]
CY = [0, 0, 0, 1, -1, 1, -1, -1, 1]


@pytest.mark.parametrize("name", ["naca2412-3lvl", "naca0012-6lvl", "two-loops-periodic-3lvl"])
def test_flag_words_encode_the_tables(name):
    # the flag word the level kernel reads, decoded and checked against the cell codes, the
    # cut links and the band / coalescence rules restated here (reading of the Rohde
    # transfers: band = active cells beside a covered cell; pulled direction d of a band
    # cell coalesces iff c - c_d, c - (c_dx, 0) or c - (0, c_dy) is covered)
    cfg, loops = CASES[name]()
    g = pkg.Solver(cfg, host_only=True)
    g.set_geometry(loops)
    L = cfg["levels"]
    ijd, _ = g.cut_links()
    for l in range(L):
        i0, j0, nx, ny = g.level_box(l)
        f = g.flags(l).astype(np.int64)
        m = g.mask(l)
        kind = f & 3
        solid = (f >> 2) & 1
        # cells without a slot: absent ones, and on finer levels the solid cells of tiles
        # that hold nothing else (no state is kept for them)
        slot = f != 0
        assert np.all(m[~slot] == 0) if l == 0 else np.all(np.isin(m[~slot], (0, 5)))
        assert np.array_equal(solid[slot] == 1, m[slot] == 5)
        code = {1: 1, 2: 1, 3: 2, 4: 3}
        for c, k in code.items():
            assert np.all(kind[m == c] == k), (l, c)
        assert np.array_equal((f >> 4) & 1 == 1, m == 2)
        # band and coalescence, with kinds padded by absent cells around the box; checked
        # where every cell they look at has a known kind
        K = np.zeros((ny + 2, nx + 2), dtype=np.int64)
        K[1:-1, 1:-1] = kind
        known = np.ones((ny + 2, nx + 2), dtype=bool)
        known[1:-1, 1:-1] = slot | (m == 0)
        cov = K == 2
        near_cov = np.zeros((ny, nx), dtype=bool)
        seen = np.ones((ny, nx), dtype=bool)
        for d in range(1, 9):
            near_cov |= cov[1 + CY[d]:1 + CY[d] + ny, 1 + CX[d]:1 + CX[d] + nx]
            seen &= known[1 + CY[d]:1 + CY[d] + ny, 1 + CX[d]:1 + CX[d] + nx]
        seen &= slot
        band = (f >> 3) & 1
        if not (l == 0 and cfg.get("periodic")):
            assert np.array_equal((band == 1)[seen], ((kind == 1) & near_cov)[seen]), l
        coal = (f >> 5) & 0xFF
        want = np.zeros((ny, nx), dtype=np.int64)
        for d in range(1, 9):
            hit = np.zeros((ny, nx), dtype=bool)
            for sx, sy in ((CX[d], CY[d]), (CX[d], 0), (0, CY[d])):
                hit |= cov[1 - sy:1 - sy + ny, 1 - sx:1 - sx + nx]
            want |= np.where(hit & (band == 1), 1 << (d - 1), 0)
        assert np.array_equal(coal[seen], want[seen]), l
        assert np.all(coal[band == 0] == 0)
        # bits 13..20: cut links of boundary nodes (finest level only, as listed by
        # lbm_get_cut_links); on ghosts, the directions whose upstream cell is not an active or
        # ghost fluid cell (the ghost keeps its own value there); on band cells, the children
        # (b * 2 + a) that are solid or have no slot on the next level
        hi = (f >> 13) & 0xFF
        want = np.zeros((ny, nx), dtype=np.int64)
        if l == L - 1:
            for i, j, d in ijd:
                want[j - j0, i - i0] |= 1 << (d - 1)
        ghost = kind == 3
        S = np.ones((ny + 2, nx + 2), dtype=bool)
        S[1:-1, 1:-1] = solid == 1
        flows = ((K == 1) | (K == 3)) & ~S
        for d in range(1, 9):
            up = flows[1 - CY[d]:1 - CY[d] + ny, 1 - CX[d]:1 - CX[d] + nx]
            want |= np.where(ghost & ~up, 1 << (d - 1), 0)
        if l < L - 1:
            fi0, fj0, fnx, fny = g.level_box(l + 1)
            ff = g.flags(l + 1).astype(np.int64)
            fm = g.mask(l + 1)
            for j, i in zip(*np.nonzero(band == 1)):
                for m_ in range(4):
                    ci, cj = 2 * (i + i0) + (m_ & 1) - fi0, 2 * (j + j0) + (m_ >> 1) - fj0
                    inside = 0 <= ci < fnx and 0 <= cj < fny
                    if not inside or ff[cj, ci] == 0 or fm[cj, ci] == 5:
                        want[j, i] |= 1 << m_
        assert np.array_equal(hi, want), l
        # level-0 edges of a box with domain boundaries, and the column before the outlet
        edges = (f >> 21) & 0x1F
        if l == 0 and not cfg.get("periodic"):
            I, J = np.meshgrid(np.arange(i0, i0 + nx), np.arange(j0, j0 + ny))
            pres = kind != 0
            want = ((I == 0) * 1 + (I == cfg["nx0"] - 1) * 2 + (J == 0) * 4 + (J == cfg["ny0"] - 1) * 8 +
                    (I == cfg["nx0"] - 2) * 16) * pres
            assert np.array_equal(edges, want)
        else:
            assert np.all(edges == 0)
    g.close()
