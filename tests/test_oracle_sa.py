"""Pins of the oracle's SA-neg model (Sec 2.2, eqs 11-17) and its explicit
finite-difference update (Lax-Wendroff convection, centred diffusion, LSQ vorticity)."""
import math

import numpy as np
import pytest

import oracle

KAPPA, CB1, CB2, SIGMA, CV1 = 0.41, 0.1355, 0.622, 2.0 / 3.0, 7.1
CX = np.array([0, 1, -1, 0, 0, 1, -1, 1, -1])
CY = np.array([0, 0, 0, 1, -1, 1, -1, -1, 1])
FAR = 1e12


def eq21(yp):
    k3 = (KAPPA * yp) ** 3
    return (CV1**3 + k3) / (CV1**3 + k3 * (1.0 + KAPPA * yp))


@pytest.mark.parametrize("yp", [0.1, 1.0, 4.0, 10.0, 30.0, 100.0, 1e3, 1e4])
def test_law_of_the_wall_balance(yp):
    # With chi = kappa y+ and du/dy from eq 21 (eq 20 solution), production - destruction must
    # balance the diffusion term (1/sigma)[d/dy((nu+nt)dnt/dy) + cb2 (dnt/dy)^2] = kappa^2 ut^2 (1+cb2)/sigma
    # exactly, at every y+ (pins fv1, fv2, the S_bar reading, S_tilde, r, g, fw and cw1).
    nu, ut = 1.5e-5, 0.05
    y = yp * nu / ut
    vort = ut * ut / nu * eq21(yp)
    P, D = oracle.sa_source(KAPPA * yp, nu, vort, y)
    diff = KAPPA**2 * ut**2 * (1 + CB2) / SIGMA
    assert (P - D + diff) / diff == pytest.approx(0.0, abs=1e-12)


def test_modified_vorticity_stays_positive_and_continuous():
    # eq 14 second branch (S_bar < -cv2 Omega) must keep S_tilde positive ("defined to be positive")
    # and meet the first branch continuously at S_bar = -cv2 Omega (reading cv3 = 0.9)
    nu, chi = 1e-3, 5.0                       # fv2 < 0 at chi = 5
    vort = 1.0
    fv1 = chi**3 / (chi**3 + CV1**3)
    fv2 = 1 - chi / (1 + chi * fv1)
    st_prev = None
    for ratio in np.linspace(-0.05, -3.0, 300):      # S_bar / Omega
        d = math.sqrt(chi * nu * fv2 / (KAPPA**2 * ratio * vort))
        P, _ = oracle.sa_source(chi, nu, vort, d)
        st = P / (CB1 * chi * nu)
        assert st > 0
        assert st < vort * 1.000001
        if st_prev is not None:
            assert abs(st - st_prev) < 0.05 * vort
        st_prev = st
    # continuity at the switch point
    for eps in (1e-7, -1e-7):
        r = -0.7 + eps
        d = math.sqrt(chi * nu * fv2 / (KAPPA**2 * r * vort))
        P, _ = oracle.sa_source(chi, nu, vort, d)
        assert P / (CB1 * chi * nu) == pytest.approx(0.3 * vort, abs=1e-5)


def test_negative_branch_continuous_at_zero():
    nu, vort, d = 1e-5, 0.3, 2.0
    for eps in (1e-12, -1e-12):
        P, D = oracle.sa_source(eps, nu, vort, d)
        assert abs(P - D) < 1e-15
    # SA-neg production is positive for negative nu_t~ (drives it back towards zero), eq 17
    P, D = oracle.sa_source(-0.5, nu, vort, d)
    assert P > 0 and D < 0


def _stencil(fun):
    return np.array([fun(CX[k], CY[k]) for k in range(9)], dtype=np.float64)


@pytest.mark.parametrize("u,v", [(0.3, 0.0), (0.0, -0.2), (0.25, 0.15), (-0.4, 0.3)])
def test_lax_wendroff_translates_quadratics_exactly(u, v):
    # a second-order Taylor (Lax-Wendroff) step advects any quadratic field exactly; nu -> 0 removes
    # diffusion (it scales as nu^2 against nu for convection) and d -> inf removes the sources
    c = [1.3, 0.2, -0.35, 0.07, -0.04, 0.11]
    q = lambda x, y: c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * x * y + c[5] * y * y
    chi = _stencil(q)
    new = oracle.sa_update_point(chi, np.full(9, u), np.full(9, v), FAR, 1e-14)
    assert new == pytest.approx(q(-u, -v), rel=1e-9)


@pytest.mark.parametrize("grad", [(0.01, -0.02, 0.03, 0.005), (0.0, 0.05, -0.02, 0.0), (-0.03, 0.0, 0.0, 0.04)])
def test_lsq_vorticity_exact_for_linear_velocity(grad):
    # uniform chi: no convection or diffusion; the update is cb1 * Omega * chi with Omega = |dv/dx - du/dy|
    a, b, c, e = grad
    ux = _stencil(lambda x, y: 0.1 + a * x + b * y)
    uy = _stencil(lambda x, y: -0.05 + c * x + e * y)
    # constant velocity offset is removed from convection because chi is uniform
    chi0 = 2.0
    nu = 1e-6
    new = oracle.sa_update_point(np.full(9, chi0), ux, uy, FAR, nu)
    # the diffusion's diagonal is implicit: the source enters divided by 1 + sum_f D_f / sigma
    a = 4.0 * nu * (1.0 + chi0) / SIGMA
    assert (new - chi0) * (1.0 + a) / (CB1 * chi0) == pytest.approx(abs(c - b), rel=1e-9, abs=1e-15)


def test_diffusion_second_order():
    # u = 0, d -> inf: the update equals (1/sigma)[div((nu+nt) grad nt) + cb2 |grad nt|^2] up to O(h^2)
    nu = 1.0
    errs = []
    for h in (0.2, 0.1, 0.05):
        f = lambda x, y: 1.0 + 0.5 * math.sin(0.7 + x) * math.cos(0.3 + 2 * y)
        chi = _stencil(lambda i, j: f(i * h, j * h))
        new = oracle.sa_update_point(chi, np.zeros(9), np.zeros(9), FAR, nu)
        # the diagonal of the diffusion is implicit: the increment is the explicit one
        # divided by 1 + sum_f D_f / sigma, D_f the face means of nu + nu~ (nu~ = chi nu)
        D = nu * (1.0 + chi)
        a = sum(0.5 * (D[0] + D[k]) for k in (1, 2, 3, 4)) / SIGMA
        # analytic right-hand side in physical units, scaled by h^2 for the unit lattice
        x, y = 0.0, 0.0
        nt = f(x, y)
        fx = 0.5 * math.cos(0.7 + x) * math.cos(0.3 + 2 * y)
        fy = -1.0 * math.sin(0.7 + x) * math.sin(0.3 + 2 * y)
        fxx = -0.5 * math.sin(0.7 + x) * math.cos(0.3 + 2 * y)
        fyy = -2.0 * math.sin(0.7 + x) * math.cos(0.3 + 2 * y)
        rhs = ((1 + nt) * (fxx + fyy) + (fx * fx + fy * fy) + CB2 * (fx * fx + fy * fy)) / SIGMA
        errs.append(abs((new - chi[0]) * (1.0 + a) / h**2 - rhs))
    assert math.log2(errs[0] / errs[1]) > 1.8
    assert math.log2(errs[1] / errs[2]) > 1.8


def _stencil(fn):
    return np.array([fn(cx, cy) for cx, cy in zip(CX, CY)], dtype=np.float64)


@pytest.mark.parametrize("u", [0.1, -0.1])
def test_upwind_convection_takes_the_upstream_difference(u):
    # first-order upwind (Sec 3.3) on phi = x^2: -u (phi_0 - phi_W) = u for u > 0 and
    # -u (phi_E - phi_0) = -u for u < 0, i.e. +0.1 both times; Lax-Wendroff gives u^2 = 0.01
    phi = _stencil(lambda x, y: float(x * x))
    assert oracle.sa_convection(phi, u, 0.0, 1) == pytest.approx(0.1, abs=1e-15)
    assert oracle.sa_convection(phi, u, 0.0, 0) == pytest.approx(0.01, abs=1e-15)
    phi_y = _stencil(lambda x, y: float(y * y))
    assert oracle.sa_convection(phi_y, 0.0, u, 1) == pytest.approx(0.1, abs=1e-15)


def test_upwind_is_exact_for_linear_fields_and_monotone():
    rng = np.random.default_rng(5)
    for _ in range(200):
        a, b, c = rng.normal(size=3)
        u, v = rng.uniform(-0.5, 0.5, size=2)
        lin = _stencil(lambda x, y: a + b * x + c * y)
        assert oracle.sa_convection(lin, u, v, 1) == pytest.approx(-(u * b + v * c), abs=1e-13)
        # |u| + |v| <= 1: the updated value is a convex combination of the centre and its
        # upstream neighbours, so it stays inside their range
        phi = rng.normal(size=9)
        new = phi[0] + oracle.sa_convection(phi, u, v, 1)
        ups = [phi[0], phi[2] if u > 0 else phi[1], phi[4] if v > 0 else phi[3]]
        assert min(ups) - 1e-13 <= new <= max(ups) + 1e-13


def test_sa_update_uses_the_requested_convection():
    chi = _stencil(lambda x, y: 3.0 + 0.2 * x * x)
    u9, v9 = np.full(9, 0.1), np.zeros(9)
    nu = 1e-14                                   # diffusion and sources vanish with nu
    lw = oracle.sa_update_point(chi, u9, v9, FAR, nu, 0)
    up = oracle.sa_update_point(chi, u9, v9, FAR, nu, 1)
    assert lw - 3.0 == pytest.approx(0.5 * 0.01 * 0.4, rel=1e-9)
    assert up - 3.0 == pytest.approx(-0.1 * (0.0 - 0.2), rel=1e-9)


def _sliver_case():
    """Periodic 32 x 32 box (one level) with a wall sliver 0.004 cells thick lying 0.003-0.007
    cells above the row of cell centres y = 16.5: no centre is inside it, so no link is cut and
    the sixteen nodes beside it are plain fluid nodes at d < 1/2 from the wall."""
    from paper_2601_18443_gb300 import workloads as W

    cfg = W.base_config(levels=1, nx0=32, ny0=32, periodic=1, solid_walls=1, turbulence=1, wall_model=0, Re=100.0)
    sliver = np.array([[8.0, 16.505], [24.0, 16.503], [24.0, 16.507]])
    return cfg, [sliver]


def test_sa_sees_at_least_half_a_spacing_of_wall_distance():
    # From a uniform state the first SA-neg update of every node is the point update of a
    # uniform stencil; beside the sliver it must be taken at d = 1/2, elsewhere at the node's d
    cfg, loops = _sliver_case()
    r = oracle.Solver(cfg)
    r.set_geometry(loops)
    assert len(r.cut_links()[0]) == 0
    d = r.wall_distance(0)
    f0 = r.get_fields(0)
    U = f0["ux"][0, 0]
    assert np.all(f0["chi"] == 3.0) and np.all(f0["ux"] == U) and np.all(f0["uy"] == 0.0)
    nu = cfg["Ma"] * math.sqrt(1.0 / 3.0) / cfg["Re"]
    r.step(1)
    chi1 = r.get_fields(0)["chi"]
    ch, u, v = np.full(9, 3.0), np.full(9, U), np.zeros(9)
    near = d < 0.5
    assert near.sum() == 16
    for j, i in zip(*np.nonzero(np.ones_like(d, dtype=bool))):
        want = oracle.sa_update_point(ch, u, v, max(d[j, i], 0.5), nu)
        assert chi1[j, i] == pytest.approx(want, rel=1e-14, abs=1e-14)
    # the update at the true distance would have driven nu~ far below zero in one step
    j, i = np.argwhere(near)[0]
    assert oracle.sa_update_point(ch, u, v, d[j, i], nu) < -100.0
    assert chi1[near].min() > 2.5


def test_sliver_run_stays_finite_and_the_flow_uniform():
    # no cut links: the populations stay at the uniform equilibrium whatever nu_t does, and
    # nu~ stays bounded beside the sliver over many steps
    cfg, loops = _sliver_case()
    r = oracle.Solver(cfg)
    r.set_geometry(loops)
    r.step(300)
    f = r.get_fields(0)
    assert np.all(np.isfinite(f["chi"]))
    assert np.abs(f["ux"] - f["ux"][0, 0]).max() < 1e-15 and np.abs(f["uy"]).max() < 1e-15
    assert f["chi"].min() > 0.0 and f["chi"].max() <= 3.0 + 1e-12


def test_implicit_diagonal_keeps_the_diffusion_a_weighted_mean():
    # nu~ so large that explicit diffusion (factor (nu + nu~)/sigma per step, well above 1/4)
    # would overshoot: with the diagonal implicit, a stencil without source, convection or
    # cb2 term (gradient zero by symmetry) updates to a weighted mean of its values
    nu = 1e-3
    chi = np.array([5.0e4, 9.0e4, 9.0e4, 2.0e4, 2.0e4, 7.0e4, 7.0e4, 7.0e4, 7.0e4])
    new = oracle.sa_update_point(chi, np.zeros(9), np.zeros(9), FAR, nu)
    assert chi.min() <= new <= chi.max()
    D = nu * (1.0 + chi)
    Df = [0.5 * (D[0] + D[k]) for k in (1, 2, 3, 4)]
    explicit = chi[0] + sum(f * (chi[k] - chi[0]) for f, k in zip(Df, (1, 2, 3, 4))) / SIGMA
    assert not (chi.min() <= explicit <= chi.max())      # the explicit step leaves the range
    # and the same fixed point: a stencil in balance does not move
    flat = np.full(9, 7.0e4)
    assert oracle.sa_update_point(flat, np.zeros(9), np.zeros(9), FAR, nu) == pytest.approx(7.0e4, rel=1e-14)
