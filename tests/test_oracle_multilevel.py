"""Pins of the oracle's Rohde explosion/coalescence with 2:1 sub-cycling (Sec 2.1):
strict mass conservation across level interfaces (the paper's stated property), momentum
conservation, and exactness of a uniform stream through refined patches."""
import math

import numpy as np
import pytest

import oracle
from paper_2601_18443_gb300 import workloads as W

U_LAT = 0.1 * math.sqrt(1.0 / 3.0)

PATCHES = {
    "square-2lvl": ([W.rectangle(12, 12, 20, 20)], 2, 32),
    "square-3lvl": ([W.rectangle(21, 21, 27, 27)], 3, 48),
    "L-2lvl": ([W.l_shape(10, 10, 22, 22, 16, 16)], 2, 32),
    "diamond-3lvl": ([np.array([[24.0, 14.0], [34.0, 24.0], [24.0, 34.0], [14.0, 24.0]])], 3, 48),
    "two-patches-3lvl": ([W.rectangle(10, 10, 15, 15), W.rectangle(30, 28, 36, 31)], 3, 48),
}


def _solver(loops, levels, n, seed=1):
    cfg = W.base_config(levels=levels, nx0=n, ny0=n, h0=1.0, Re=U_LAT / 0.02, Ma=0.1, periodic=1, solid_walls=0,
                        layers=3, wall_model=3)
    s = oracle.Solver(cfg)
    s.set_geometry(loops)
    rng = np.random.default_rng(seed)
    k = 2 * np.pi / n
    for l in range(levels):
        i0, j0, nx, ny = s.level_box(l)
        x = (np.arange(i0, i0 + nx) + 0.5) / 2**l
        y = (np.arange(j0, j0 + ny) + 0.5) / 2**l
        X, Y = np.meshgrid(x, y)
        ux = 0.02 * np.sin(k * X) * np.cos(k * Y) + 0.01 + 0.002 * rng.standard_normal(X.shape)
        uy = -0.02 * np.cos(k * X) * np.sin(k * Y) + 0.002 * rng.standard_normal(X.shape)
        s.set_fields(l, rho=1 + 0.001 * rng.standard_normal(X.shape), ux=ux, uy=uy)
    return s


def _momentum(s, levels):
    px = py = 0.0
    for l in range(levels):
        F = s.get_fields(l)
        a = F["mask"] == 1
        w = 4.0 ** (levels - 1 - l)
        px += w * np.sum((F["rho"] * F["ux"])[a])
        py += w * np.sum((F["rho"] * F["uy"])[a])
    return px, py


@pytest.mark.parametrize("name", list(PATCHES))
def test_mass_and_momentum_conserved(name):
    loops, levels, n = PATCHES[name]
    s = _solver(loops, levels, n)
    for l in range(1, levels):
        assert (s.get_fields(l)["mask"] == 4).sum() > 0      # interfaces exist
    m0, p0 = s.mass(), _momentum(s, levels)
    s.step(150)
    p1 = _momentum(s, levels)
    assert abs(s.mass() / m0 - 1) < 1e-13
    assert abs(p1[0] - p0[0]) / abs(p0[0]) < 1e-12
    assert abs(p1[1] - p0[1]) / abs(p0[0]) < 1e-12


def test_uniform_stream_through_patches_stays_uniform():
    loops, levels, n = PATCHES["diamond-3lvl"]
    cfg = W.base_config(levels=levels, nx0=n, ny0=n, h0=1.0, Re=U_LAT / 0.01, Ma=0.1, periodic=1, solid_walls=0,
                        layers=3, wall_model=3, turbulence=1)
    s = oracle.Solver(cfg)
    s.set_geometry(loops)
    for l in range(levels):
        i0, j0, nx, ny = s.level_box(l)
        s.set_fields(l, rho=np.full((ny, nx), 1.0), ux=np.full((ny, nx), 0.04), uy=np.full((ny, nx), -0.025))
    s.step(60)
    for l in range(levels):
        F = s.get_fields(l)
        a = F["mask"] == 1
        assert np.abs(F["ux"][a] - 0.04).max() < 1e-14
        assert np.abs(F["uy"][a] + 0.025).max() < 1e-14
        assert np.abs(F["rho"][a] - 1.0).max() < 1e-14
        assert np.abs(F["chi"][a] - 3.0).max() < 1e-12


def test_taylor_green_across_a_refined_patch():
    # a refined patch must not spoil the decay rate (first order in time at the interface, O6)
    nu, U0, n = 0.05, 1e-3, 32
    res = []
    for loops, levels in (([], 1), ([W.rectangle(13, 13, 19, 19)], 2)):
        cfg = W.base_config(levels=levels, nx0=n, ny0=n, h0=1.0, Re=U_LAT / nu, Ma=0.1, periodic=1,
                            solid_walls=0, layers=3, wall_model=3)
        s = oracle.Solver(cfg)
        s.set_geometry(loops)
        k = 2 * np.pi / n
        for l in range(levels):
            i0, j0, nx, ny = s.level_box(l)
            x = (np.arange(i0, i0 + nx) + 0.5) / 2**l
            y = (np.arange(j0, j0 + ny) + 0.5) / 2**l
            X, Y = np.meshgrid(x, y)
            s.set_fields(l, rho=np.ones_like(X), ux=-U0 * np.cos(k * X) * np.sin(k * Y),
                         uy=U0 * np.sin(k * X) * np.cos(k * Y))
        T = int(0.5 / (2 * nu * k * k))
        s.step(T // 2)
        e1 = s.get_fields(0)["uy"]
        s.step(T // 2)
        e2 = s.get_fields(0)["uy"]
        a = s.get_fields(0)["mask"] == 1
        res.append(math.log((e1[a] ** 2).sum() / (e2[a] ** 2).sum()) / (2 * (T // 2)) / (2 * nu * k * k) - 1)
    assert abs(res[0]) < 2e-3
    assert abs(res[1]) < 2e-2


# --------------------------------------------------------------------------- interface fields (Sec 2.2)
# The ghost children of a band cell get chi and u from a linear least-squares fit over the
# band cell's D2Q9 neighbourhood, evaluated at the child centre (offsets of a quarter of the
# parent spacing); rho is copied from the parent.  A covered parent gets the mean rho and chi
# of its fluid children and their mass-weighted velocity.  Linear fields pin both: the fit
# reproduces a linear field exactly, and the mean of a linear field over the four children
# is its value at the parent centre.

LIN = dict(chi=(2.0, 0.031, -0.017), ux=(0.03, 2.5e-3, 1.5e-3), uy=(-0.01, -1e-3, 3e-3), rho=(1.0, 4e-3, -3e-3))


def _lin(key, X, Y):
    a, b, c = LIN[key]
    return a + b * X + c * Y


def _centres(s, l):
    """Cell centres of level l in level-0 lattice units (h0 = 1, origin 0)."""
    i0, j0, nx, ny = s.level_box(l)
    x = (np.arange(i0, i0 + nx) + 0.5) / 2**l
    y = (np.arange(j0, j0 + ny) + 0.5) / 2**l
    return np.meshgrid(x, y)


def _linear_solver(loops, levels, n, rho_linear, solid_walls=0, periodic=1):
    cfg = W.base_config(levels=levels, nx0=n, ny0=n, h0=1.0, Re=U_LAT / 0.02, Ma=0.1, periodic=periodic,
                        solid_walls=solid_walls, layers=3, wall_model=3, turbulence=1)
    s = oracle.Solver(cfg)
    s.set_geometry(loops)
    for l in range(levels):
        X, Y = _centres(s, l)
        rho = _lin("rho", X, Y) if rho_linear else np.ones_like(X)
        s.set_fields(l, rho=rho, ux=_lin("ux", X, Y), uy=_lin("uy", X, Y), chi=_lin("chi", X, Y))
    return s


@pytest.mark.parametrize("name", ["square-2lvl", "square-3lvl", "L-2lvl", "diamond-3lvl", "two-patches-3lvl"])
def test_ghost_fields_reproduce_a_linear_field(name):
    loops, levels, n = PATCHES[name]
    s = _linear_solver(loops, levels, n, rho_linear=False)
    for l in range(1, levels):
        F = s.get_fields(l)
        g = F["mask"] == 4
        assert g.sum() > 0
        X, Y = _centres(s, l)
        for key in ("chi", "ux", "uy"):
            err = np.abs(F[key][g] - _lin(key, X, Y)[g]).max()
            assert err < 1e-13, (l, key, err)
        assert np.abs(F["rho"][g] - 1.0).max() < 1e-15


def test_ghost_density_is_the_parent_density():
    loops, levels, n = PATCHES["square-2lvl"]
    s = _linear_solver(loops, levels, n, rho_linear=True)
    P, F = s.get_fields(0), s.get_fields(1)
    i0p, j0p = s.level_box(0)[:2]
    i0f, j0f = s.level_box(1)[:2]
    jj, ii = np.nonzero(F["mask"] == 4)
    parent = P["rho"][(jj + j0f) // 2 - j0p, (ii + i0f) // 2 - i0p]
    assert np.array_equal(F["rho"][jj, ii], parent)


@pytest.mark.parametrize("name", ["square-2lvl", "square-3lvl", "L-2lvl", "diamond-3lvl"])
def test_covered_cells_hold_the_parent_centre_values(name):
    # constant density: the mass weighting is a plain mean, so every restricted field of a
    # linear state is its value at the parent centre
    loops, levels, n = PATCHES[name]
    s = _linear_solver(loops, levels, n, rho_linear=False)
    for l in range(levels - 1):
        F = s.get_fields(l)
        c = F["mask"] == 3
        assert c.sum() > 0
        X, Y = _centres(s, l)
        for key in ("chi", "ux", "uy"):
            err = np.abs(F[key][c] - _lin(key, X, Y)[c]).max()
            assert err < 1e-13, (l, key, err)


def test_covered_velocity_is_mass_weighted():
    # linear rho and u on two levels: the covered parent holds rho and chi at its centre and
    # u = sum_c rho_c u_c / sum_c rho_c over its four children, which differs from the plain
    # mean by about 3e-7 here (far above the rounding of the sums)
    loops, levels, n = PATCHES["square-2lvl"]
    s = _linear_solver(loops, levels, n, rho_linear=True)
    F = s.get_fields(0)
    c = F["mask"] == 3
    X, Y = _centres(s, 0)
    for key in ("rho", "chi"):
        assert np.abs(F[key][c] - _lin(key, X, Y)[c]).max() < 1e-14
    off = [(-0.25, -0.25), (0.25, -0.25), (-0.25, 0.25), (0.25, 0.25)]
    rho_c = [_lin("rho", X + a, Y + b) for a, b in off]
    for key in ("ux", "uy"):
        mw = sum(r * _lin(key, X + a, Y + b) for r, (a, b) in zip(rho_c, off)) / sum(rho_c)
        plain = _lin(key, X, Y)
        assert np.abs(mw - plain)[c].min() > 1e-7          # the weighting is visible
        assert np.abs(F[key][c] - mw[c]).max() < 1e-15, key


def test_restriction_skips_solid_children():
    # a wall inside the refined patch: covered parents with solid children hold the mean over
    # their fluid children only (rho, chi) and the mass-weighted velocity over them
    n = 32
    cfg = W.base_config(levels=2, nx0=n, ny0=n, h0=1.0, Re=U_LAT / 0.02, Ma=0.1, periodic=1, solid_walls=1,
                        layers=3, wall_model=3, turbulence=1)
    s = oracle.Solver(cfg)
    s.set_geometry([np.array([[13.3, 12.2], [19.1, 13.7], [17.6, 19.4], [12.4, 17.9]])])
    for l in range(2):
        X, Y = _centres(s, l)
        s.set_fields(l, rho=_lin("rho", X, Y), ux=_lin("ux", X, Y), uy=_lin("uy", X, Y), chi=_lin("chi", X, Y))
    P, F = s.get_fields(0), s.get_fields(1)
    i0p, j0p = s.level_box(0)[:2]
    i0f, j0f = s.level_box(1)[:2]
    XF, YF = _centres(s, 1)
    partial = 0
    for j, i in zip(*np.nonzero(P["mask"] == 3)):
        gi, gj = i + i0p, j + j0p
        kids = [(2 * gj + b - j0f, 2 * gi + a - i0f) for b in (0, 1) for a in (0, 1)]
        fluid = [(y, x) for y, x in kids if F["mask"][y, x] != 5]
        if not fluid:
            continue
        partial += len(fluid) < 4
        r = np.array([_lin("rho", XF[y, x], YF[y, x]) for y, x in fluid])
        want = {"rho": r.mean(), "chi": np.mean([_lin("chi", XF[y, x], YF[y, x]) for y, x in fluid])}
        for key in ("ux", "uy"):
            want[key] = np.sum(r * np.array([_lin(key, XF[y, x], YF[y, x]) for y, x in fluid])) / r.sum()
        for key, v in want.items():
            assert abs(P[key][j, i] - v) < 1e-14, (key, i, j)
    assert partial > 0
