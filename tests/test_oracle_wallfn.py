"""Pins of the oracle's analytical SA wall function (Sec 2.2, eqs 20-22) and its
inversion (Sec 2.3 step 3)."""
import math

import numpy as np
import pytest

import oracle

KAPPA = 0.41          # Sec 2.2 constants
CV1 = 7.1
CV1_3 = CV1**3


def eq21(yp):
    """du+/dy+ as printed in eq 21 (independent of the eq 22 fit constants)."""
    k3 = (KAPPA * yp) ** 3
    return (CV1**3 + k3) / (CV1**3 + k3 * (1.0 + KAPPA * yp))


def test_wall_value_near_zero():
    # law of the wall: u+ -> 0 at the wall; the published fit gives 5.18e-4
    assert abs(oracle.wf_uplus(0.0)) < 6e-4
    assert oracle.wf_uplus(0.0) == pytest.approx(5.179e-4, abs=2e-6)


@pytest.mark.parametrize("yp", [0.05, 0.5, 3.0, 6.5, 6.93, 7.4, 15.0, 60.0, 400.0, 3e3, 5e4])
def test_slope_matches_eq21(yp):
    # derivative of the eq 22 fit (central differences) equals eq 21: pins all nine constants
    h = 1e-5 * max(1.0, yp)
    d = (oracle.wf_uplus(yp + h) - oracle.wf_uplus(yp - h)) / (2 * h)
    assert d == pytest.approx(eq21(yp), rel=2e-7, abs=1e-9)
    assert oracle.wf_dudy(yp) == pytest.approx(eq21(yp), rel=1e-14)


def test_continuous_branch_at_minus_a2():
    # the literal arctan(b/(y+ + a2)) jumps by c4*pi at y+ = -a2; the reading atan2 is continuous
    a2 = 6.9287093849022945
    lo, hi = oracle.wf_uplus(a2 - 1e-9), oracle.wf_uplus(a2 + 1e-9)
    assert abs(hi - lo) < 1e-8


def test_log_law_asymptote():
    # far from the wall u+ - ln(y+)/kappa -> B (2(c1-c2) = 1/kappa, arctangents -> 0)
    vals = [oracle.wf_uplus(y) - math.log(y) / KAPPA for y in (1e6, 1e7, 1e8, 1e9)]
    assert np.ptp(vals) < 1e-5
    assert vals[-1] == pytest.approx(5.033908790505579, abs=1e-6)


def test_viscous_sublayer():
    for yp in (0.1, 0.3, 1.0):
        assert oracle.wf_uplus(yp) == pytest.approx(yp, abs=2e-3)


@pytest.mark.parametrize("yp", [0.1, 1.0, 5.0, 11.0, 30.0, 100.0, 1e3, 1e4, 1e5])
def test_inversion_recovers_utau(yp):
    nu, y = 1.5e-5, 2.0
    ut = yp * nu / y
    u = ut * oracle.wf_uplus(yp)
    assert oracle.wf_utau(u, y, nu) == pytest.approx(ut, rel=1e-12)


def test_inversion_zero_velocity():
    assert oracle.wf_utau(0.0, 2.0, 1e-5) == 0.0


def test_nishimura_slip_follows_eq31():
    # Sec 3.1.5, eq 31: u_W = u_R - u_tau^2 d_WR / (nu + nu_t)|_R with d_WR = 1.75 and the SA
    # log-layer eddy viscosity (nu_t)_R = nu kappa y+_R (eq 20).  Above the flat top of a plate
    # a linear velocity profile makes the LSQ value at R exact; u_tau comes from eq 22 at R.
    from paper_2601_18443_gb300 import workloads as W
    nx0, ny0, top = 48, 32, 12.375
    nu_lat = 0.01
    U = 0.1 * math.sqrt(1.0 / 3.0)
    cfg = W.base_config(levels=1, nx0=nx0, ny0=ny0, h0=1.0, Re=U / nu_lat, Ma=0.1, wall_model=1,
                        turbulence=1, d_wr=1.75)
    s = oracle.Solver(cfg)
    s.set_geometry([W.rectangle(8.0, 6.0, 40.0, top)])
    y = np.arange(ny0) + 0.5
    a, b, chi = 0.004, 0.003, 4.0
    ux = np.tile((a + b * (y - top))[:, None], (1, nx0))
    s.set_fields(0, rho=np.ones((ny0, nx0)), ux=ux, uy=np.zeros((ny0, nx0)), chi=np.full((ny0, nx0), chi))
    ij, geo, ns = s.wall_records()
    st = s.wall_state()
    # records on the top face, away from the corners (their stencils see only the profile)
    sel = (geo[:, 3] > 0.999) & (ij[:, 0] > 12) & (ij[:, 0] < 36)
    assert sel.sum() >= 20
    for r in np.nonzero(sel)[0]:
        uR = a + b * (geo[r, 6] - top)              # R y in lattice units from the box origin
        utau = oracle.wf_utau(uR, 1.75, nu_lat)
        expect = uR - utau**2 * 1.75 / (nu_lat * (1.0 + KAPPA * utau * 1.75 / nu_lat))
        assert st[r, 3] == pytest.approx(utau, rel=1e-12)
        assert st[r, 1] == pytest.approx(expect, rel=1e-9, abs=1e-15)
        assert st[r, 2] == pytest.approx(0.0, abs=1e-12)


@pytest.mark.parametrize("nu_lat", [0.01, 2e-7])
def test_virtual_node_slip_follows_eq28(nu_lat):
    # Sec 2.3 steps 3-5: u_tau from eq 22 at R (d_WR = 2), u_V = u_tau u+(y+_V) at the virtual
    # node (d_WV = 1), the slip of eq 28 u_W = u_V - u_tau^2 d_WV / (nu (1 + kappa y+_V)) along
    # t, and the Dirichlet chi_B = kappa u_tau d_WB / nu.  Linear profile above a plate top, as
    # in the eq 31 pin.  At the small viscosity y+_V is in the log layer, where eq 28 tends to
    # u_W = u_tau (u+(y+_V) - 1/kappa).
    from paper_2601_18443_gb300 import workloads as W
    nx0, ny0, top = 48, 32, 12.375
    U = 0.1 * math.sqrt(1.0 / 3.0)
    cfg = W.base_config(levels=1, nx0=nx0, ny0=ny0, h0=1.0, Re=U / nu_lat, Ma=0.1, wall_model=0,
                        turbulence=1, d_wr=2.0, d_wv=1.0)
    s = oracle.Solver(cfg)
    s.set_geometry([W.rectangle(8.0, 6.0, 40.0, top)])
    y = np.arange(ny0) + 0.5
    a, b = 0.004, 0.003
    ux = np.tile((a + b * (y - top))[:, None], (1, nx0))
    s.set_fields(0, rho=np.ones((ny0, nx0)), ux=ux, uy=np.zeros((ny0, nx0)), chi=np.full((ny0, nx0), 4.0))
    ij, geo, ns = s.wall_records()
    st = s.wall_state()
    sel = (geo[:, 3] > 0.999) & (ij[:, 0] > 12) & (ij[:, 0] < 36)
    assert sel.sum() >= 20
    n_log = 0
    for r in np.nonzero(sel)[0]:
        uR = a + b * (geo[r, 6] - top)
        utau = oracle.wf_utau(uR, 2.0, nu_lat)
        ypv = utau * 1.0 / nu_lat
        uV = utau * oracle.wf_uplus(ypv)
        uW = uV - utau**2 * 1.0 / (nu_lat * (1.0 + KAPPA * ypv))
        assert st[r, 3] == pytest.approx(utau, rel=1e-12)
        assert st[r, 1] == pytest.approx(uW, rel=1e-9, abs=1e-15)
        assert st[r, 2] == pytest.approx(0.0, abs=1e-12)
        assert st[r, 4] == pytest.approx(KAPPA * utau * geo[r, 4] / nu_lat, rel=1e-12)
        if ypv > 200.0:
            n_log += 1
            assert uW == pytest.approx(utau * (oracle.wf_uplus(ypv) - 1.0 / KAPPA), rel=2e-2)
    assert n_log == (sel.sum() if nu_lat < 1e-6 else 0)
