"""Pins of the oracle's analytical SA wall function (Sec 2.2, eqs 20-22) and its
inversion (Sec 2.3 step 3)."""
import math

import numpy as np
import pytest

import oracle

KAPPA = 0.41          # Sec 2.2 constants
CV1 = 7.1


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
