"""Solver-level pins of the oracle: domain boundary conditions, Yu's interpolated
bounce-back (eq 27) on flat walls at arbitrary q, Couette flow with an imposed slip,
the rest state, and Taylor-Green decay (the viscosity of eq 9)."""
import math

import numpy as np
import pytest

import oracle
from paper_2601_18443_gb300 import workloads as W

CS2 = 1.0 / 3.0
MA = 0.1
U_LAT = MA * math.sqrt(CS2)


def re_for(nu_lat, cells_per_chord=1.0):
    return U_LAT * cells_per_chord / nu_lat


@pytest.mark.parametrize("outlet", [0, 1])
def test_uniform_freestream_is_steady(outlet):
    # Zou-He inlet, symmetry planes and either outlet form reproduce a uniform stream exactly
    cfg = W.base_config(levels=1, nx0=40, ny0=20, h0=0.1, Re=1e5, Ma=MA, turbulence=1, wall_model=0, outlet=outlet)
    s = oracle.Solver(cfg)
    s.set_geometry([])
    s.step(100)
    F = s.get_fields(0)
    assert np.abs(F["ux"] - U_LAT).max() < 1e-13
    assert np.abs(F["uy"]).max() < 1e-13
    assert np.abs(F["rho"] - 1).max() < 1e-13
    assert np.abs(F["chi"] - 3.0).max() < 1e-12


def test_uniform_freestream_across_levels():
    # a refinement patch (loops drive refinement only) inside a box with domain BCs
    cfg = W.base_config(levels=3, nx0=40, ny0=24, h0=1.0, layers=3, Re=200.0, Ma=MA, turbulence=1,
                        wall_model=3, solid_walls=0)
    s = oracle.Solver(cfg)
    s.set_geometry([np.array([[18.0, 10.0], [23.0, 12.5], [19.0, 14.0]])])
    s.step(20)
    for l in range(3):
        F = s.get_fields(l)
        act = F["mask"] == 1
        assert np.abs(F["ux"][act] - U_LAT).max() < 1e-13
        assert np.abs(F["uy"][act]).max() < 1e-13
        assert np.abs(F["rho"][act] - 1).max() < 1e-13


def _channel(N, qb, nu, model):
    yb = 2.5 - qb
    yt = yb + N
    ny0, nx0 = int(math.ceil(yt)) + 3, 4
    cfg = W.base_config(levels=1, nx0=nx0, ny0=ny0, h0=1.0, Re=re_for(nu), Ma=MA, periodic=1, wall_model=model)
    s = oracle.Solver(cfg)
    s.set_geometry([W.rectangle(-5, -10, nx0 + 5, yb), W.rectangle(-5, yt, nx0 + 5, ny0 + 10)])
    return s, yb, ny0, nx0


# wall offsets exactly representable on the 1/4096 fixed-point grid
QS = [0.125, 0.375, 0.5, 0.8125]


@pytest.mark.parametrize("qb", QS)
def test_channel_decay_second_order(qb):
    # u = sin(pi y/H) exp(-nu (pi/H)^2 t) between no-slip walls at distance q from the nodes
    nu, U0 = 0.05, 1e-4
    errs = []
    for N in (8, 16, 32):
        s, yb, ny0, nx0 = _channel(N, qb, nu, 3)
        y = np.arange(ny0) + 0.5
        m = s.get_fields(0)["mask"]
        fl = (m == 1) | (m == 2)
        shape = np.sin(np.pi * (y - yb) / N)
        s.set_fields(0, rho=np.ones((ny0, nx0)), ux=np.where(fl, U0 * shape[:, None], 0.0), uy=np.zeros((ny0, nx0)))
        T = N * N / (nu * np.pi**2)
        s.step(int(0.3 * T))
        a1 = s.get_fields(0)["ux"][:, 0]
        n2 = int(0.3 * T)
        s.step(n2)
        a2 = s.get_fields(0)["ux"][:, 0]
        f = fl[:, 0]
        rate = math.log((a1[f] * shape[f]).sum() / (a2[f] * shape[f]).sum()) / n2
        errs.append(abs(rate / (nu * (np.pi / N) ** 2) - 1))
    assert errs[-1] < 1e-3
    assert math.log2(errs[1] / errs[2]) > 1.6


@pytest.mark.parametrize("qb", QS)
def test_couette_with_imposed_slip_is_linear(qb):
    nu, Uw, N = 0.05, 1e-3, 8
    s, yb, ny0, nx0 = _channel(N, qb, nu, 2)
    s.set_wall_slip(np.array([[0.0, 0.0], [Uw, 0.0]]))
    s.set_fields(0, rho=np.ones((ny0, nx0)), ux=np.zeros((ny0, nx0)), uy=np.zeros((ny0, nx0)))
    s.step(int(30 * N * N / nu))
    F = s.get_fields(0)
    y = np.arange(ny0) + 0.5
    fl = (F["mask"] == 1) | (F["mask"] == 2)
    exact = Uw * (y - yb) / N
    assert np.nanmax(np.abs((F["ux"] - exact[:, None])[fl])) / Uw < 2e-6
    assert np.nanmax(np.abs(F["uy"][fl])) < 1e-15


def test_rest_state_exact_for_any_q():
    # a closed curved wall at rest: Yu's scheme keeps f = w exactly for every q
    cfg = W.base_config(levels=1, nx0=24, ny0=24, h0=1.0, Re=re_for(0.1), Ma=MA, periodic=1, wall_model=3)
    s = oracle.Solver(cfg)
    s.set_geometry([W.naca_loop("2412", 1.0, chord=14.0, alpha_deg=17.0, offset=(5.0, 12.0))])
    F0 = s.get_fields(0)
    s.set_fields(0, rho=np.ones_like(F0["rho"]), ux=np.zeros_like(F0["rho"]), uy=np.zeros_like(F0["rho"]))
    q = s.cut_links()[1]
    assert q.min() < 0.2 and q.max() > 0.8
    s.step(100)
    F = s.get_fields(0)
    fl = (F["mask"] == 1) | (F["mask"] == 2)
    assert np.abs(F["ux"][fl]).max() < 1e-15
    assert np.abs(F["uy"][fl]).max() < 1e-15
    assert np.abs(F["rho"][fl] - 1).max() < 1e-14


def test_taylor_green_decay_rate():
    # u = U0 (-cos kx sin ky, sin kx cos ky) decays as exp(-2 nu k^2 t), nu = cs^2 (1/omega - 1/2);
    # the rate is measured after the start-up transient of the equilibrium initialisation
    nu, U0 = 0.1, 1e-3
    errs = []
    for N in (32, 64, 128):
        cfg = W.base_config(levels=1, nx0=N, ny0=N, h0=1.0, Re=re_for(nu), Ma=MA, periodic=1, wall_model=3,
                            solid_walls=0)
        s = oracle.Solver(cfg)
        s.set_geometry([])
        k = 2 * np.pi / N
        x = np.arange(N) + 0.5
        X, Y = np.meshgrid(x, x)
        ux, uy = -U0 * np.cos(k * X) * np.sin(k * Y), U0 * np.sin(k * X) * np.cos(k * Y)
        rho = 1 - U0**2 / (4 * CS2) * (np.cos(2 * k * X) + np.cos(2 * k * Y))
        s.set_fields(0, rho=rho, ux=ux, uy=uy)
        T = int(0.5 / (2 * nu * k * k))
        s.step(T // 2)
        e1 = (s.get_fields(0)["uy"] ** 2).sum()
        s.step(T // 2)
        e2 = (s.get_fields(0)["uy"] ** 2).sum()
        rate = math.log(e1 / e2) / (2 * (T // 2))
        errs.append(abs(rate / (2 * nu * k * k) - 1))
    assert errs[-1] < 2e-4
    assert math.log2(errs[0] / errs[1]) > 1.8 and math.log2(errs[1] / errs[2]) > 1.8


@pytest.mark.parametrize("outlet", [0, 1])
def test_outlet_closes_a_linear_density_profile(outlet):
    # Sec 3.1.1 outlet on the post-stream populations q = 2, 6, 8 entering from x = N.  From
    # f = f_eq(rho(x), 0) with rho = 1 + a x, one stream gives f_q(x) = w_q rho(x - c_qx) in
    # the interior, hence rho(x) and j_x = -a/3 there.  Yu's linear extrapolation continues
    # this exactly in the last column (rho(N-1), j_x = -a/3); the zero-gradient copy brings
    # rho(N-1) - a/6 and j_x = -a/6 (its entering populations carry rho(N-1) instead of rho(N)).
    nx, ny, a = 32, 16, 1e-3
    cfg = W.base_config(levels=1, nx0=nx, ny0=ny, h0=1.0, Re=1e3, Ma=MA, turbulence=0, wall_model=3, outlet=outlet)
    s = oracle.Solver(cfg)
    s.set_geometry([])
    X = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)[0]
    rho0 = 1.0 + a * (X - nx / 2)
    s.set_fields(0, rho=rho0, ux=np.zeros_like(X), uy=np.zeros_like(X))
    s.step(1)
    F = s.get_fields(0)
    mid = slice(2, nx - 1)
    assert np.abs(F["rho"][:, mid] - rho0[:, mid]).max() < 1e-15
    assert np.abs(F["rho"][:, mid] * F["ux"][:, mid] + a / 3).max() < 1e-16
    last = rho0[:, -1]
    want_rho, want_jx = (last, -a / 3) if outlet == 0 else (last - a / 6, -a / 6)
    assert np.abs(F["rho"][:, -1] - want_rho).max() < 1e-15
    assert np.abs(F["rho"][:, -1] * F["ux"][:, -1] - want_jx).max() < 1e-16
    assert np.abs(F["uy"]).max() < 1e-16


def _vortex_box(nx=96, ny=48, Re=2000.0, outlet=1):
    """Laminar 96 x 48 box (inlet, symmetry planes, outlet) with a Gaussian vortex of core 5
    cells and peak swirl U/2 convected by the free stream; it reaches the outlet after ~300 steps."""
    cfg = W.base_config(levels=1, nx0=nx, ny0=ny, h0=1.0, Re=Re, periodic=0, solid_walls=1, turbulence=0,
                        wall_model=3, Ma=0.1, outlet=outlet)
    r = oracle.Solver(cfg)
    r.set_geometry([])
    U = 0.1 * math.sqrt(1.0 / 3.0)
    X, Y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    xc, yc, R, G = 70.0, 24.0, 5.0, 0.5 * U
    s = ((X - xc) ** 2 + (Y - yc) ** 2) / R**2
    ux = U - G * (Y - yc) / R * np.exp(-s / 2)
    uy = G * (X - xc) / R * np.exp(-s / 2)
    r.set_fields(0, rho=1 - 1.5 * G**2 * np.exp(-s), ux=ux, uy=uy)
    return r, U


def test_vortex_leaves_through_the_outlet():
    # The zero-gradient outlet lets the vortex out: after 1200 steps the disturbance keeps
    # under 0.1% of its energy and the density is back at 1 to 1e-3.
    r, U = _vortex_box(outlet=1)
    f = r.get_fields(0)
    e0 = ((f["ux"] - U) ** 2 + f["uy"] ** 2).sum()
    r.step(1200)
    f = r.get_fields(0)
    e = ((f["ux"] - U) ** 2 + f["uy"] ** 2).sum()
    assert e < 1e-3 * e0
    assert np.abs(f["rho"] - 1).max() < 1e-3


def test_zou_he_inlet_imposes_the_velocity_exactly():
    # Sec 3.1.1: the inlet column's unknown populations are closed so that the post-stream
    # velocity there is (U, 0) whatever arrives from the interior (here the vortex state)
    r, U = _vortex_box()
    r.step(150)                     # the vortex's pressure pulse has reached the inlet by now
    for _ in range(3):
        r.step(1)
        f = r.get_fields(0)
        assert np.abs(f["uy"][:, 1]).max() > 1e-7          # the next column is disturbed ...
        assert np.abs(f["ux"][:, 0] - U).max() < 1e-14     # ... the inlet column is not
        assert np.abs(f["uy"][:, 0]).max() < 1e-14


def test_linear_outlet_amplifies_the_vortex():
    # Yu's linear extrapolation, the form Sec 3.1.1 names, does not let the same vortex out:
    # the disturbance grows past its initial energy once the vortex reaches the last columns.
    # This is why the workloads use the zero-gradient outlet (outlet = 1).
    r, U = _vortex_box(outlet=0)
    f = r.get_fields(0)
    e0 = ((f["ux"] - U) ** 2 + f["uy"] ** 2).sum()
    r.step(500)
    f = r.get_fields(0)
    e = ((f["ux"] - U) ** 2 + f["uy"] ** 2).sum()
    assert not np.isfinite(e) or e > e0
