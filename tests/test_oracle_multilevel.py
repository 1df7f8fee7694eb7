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
