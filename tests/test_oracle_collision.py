"""Pins of the oracle's equilibrium (eq 4) and central-moment collision (eqs 5-10)."""
import numpy as np
import pytest

import oracle

CX = np.array([0, 1, -1, 0, 0, 1, -1, 1, -1])
CY = np.array([0, 0, 0, 1, -1, 1, -1, -1, 1])
CS2 = 1.0 / 3.0
RNG = np.random.default_rng(7)
STATES = [(1.0, 0.0, 0.0), (1.03, 0.08, -0.05), (0.97, -0.12, 0.1), (1.0, 0.15, 0.15)]


def central_moments(f, ux, uy):
    bx, by = CX - ux, CY - uy
    return {"k00": f.sum(), "k10": (bx * f).sum(), "k01": (by * f).sum(), "k20": (bx**2 * f).sum(),
            "k02": (by**2 * f).sum(), "k11": (bx * by * f).sum(), "k21": (bx**2 * by * f).sum(),
            "k12": (bx * by**2 * f).sum(), "k22": (bx**2 * by**2 * f).sum()}


def d1q3(u):
    # one-dimensional three-velocity equilibrium with moments 1, u, u^2 + cs^2
    return {0: 1.0 - (u * u + CS2), 1: 0.5 * (u * u + CS2 + u), -1: 0.5 * (u * u + CS2 - u)}


@pytest.mark.parametrize("rho,ux,uy", STATES)
def test_feq_is_product_form(rho, ux, uy):
    # the fourth-order Hermite equilibrium with the 1/(4cs^8) reading equals the tensor product
    # of two D1Q3 equilibria (both share all nine D2Q9 moments)
    gx, gy = d1q3(ux), d1q3(uy)
    expect = np.array([rho * gx[cx] * gy[cy] for cx, cy in zip(CX, CY)])
    assert np.allclose(oracle.feq(rho, ux, uy), expect, rtol=0, atol=1e-15)


@pytest.mark.parametrize("rho,ux,uy", STATES)
def test_feq_central_moments_are_maxwellian(rho, ux, uy):
    k = central_moments(oracle.feq(rho, ux, uy), ux, uy)
    exp = {"k00": rho, "k10": 0, "k01": 0, "k20": rho * CS2, "k02": rho * CS2, "k11": 0, "k21": 0, "k12": 0,
           "k22": rho * CS2 * CS2}
    for key, v in exp.items():
        assert k[key] == pytest.approx(v, abs=1e-15), key


def _random_state():
    rho, ux, uy = 1 + 0.02 * RNG.standard_normal(), 0.1 * RNG.standard_normal(), 0.1 * RNG.standard_normal()
    f = oracle.feq(rho, ux, uy) * (1 + 0.05 * RNG.standard_normal(9))
    return f


@pytest.mark.parametrize("omega", [0.7, 1.0, 1.6, 1.9999])
def test_collision_conserves_mass_and_momentum(omega):
    for _ in range(5):
        f = _random_state()
        g = oracle.collide(f, omega)
        assert g.sum() == pytest.approx(f.sum(), abs=1e-15)
        assert (CX * g).sum() == pytest.approx((CX * f).sum(), abs=1e-15)
        assert (CY * g).sum() == pytest.approx((CY * f).sum(), abs=1e-15)


@pytest.mark.parametrize("omega", [0.5, 1.3, 1.95])
def test_collision_relaxes_central_moments(omega):
    # K = diag[1,1,1, omega_b=1, omega, omega, 1,1,1] on the basis of eq 6
    for _ in range(5):
        f = _random_state()
        rho = f.sum()
        ux, uy = (CX * f).sum() / rho, (CY * f).sum() / rho
        k, ks = central_moments(f, ux, uy), central_moments(oracle.collide(f, omega), ux, uy)
        assert ks["k20"] + ks["k02"] == pytest.approx(2 * rho * CS2, abs=1e-14)
        assert ks["k20"] - ks["k02"] == pytest.approx((1 - omega) * (k["k20"] - k["k02"]), abs=1e-14)
        assert ks["k11"] == pytest.approx((1 - omega) * k["k11"], abs=1e-14)
        for key in ("k21", "k12"):
            assert ks[key] == pytest.approx(0.0, abs=1e-14)
        assert ks["k22"] == pytest.approx(rho * CS2 * CS2, abs=1e-14)


def test_full_relaxation_gives_equilibrium():
    f = _random_state()
    rho = f.sum()
    g = oracle.collide(f, 1.0)
    assert np.allclose(g, oracle.feq(rho, (CX * f).sum() / rho, (CY * f).sum() / rho), atol=1e-15)


def test_collision_commutes_with_lattice_rotation():
    # rotation by 90 degrees: (cx, cy) -> (-cy, cx); catches index/sign errors in the lattice tables
    perm = [int(np.where((CX == -CY[i]) & (CY == CX[i]))[0][0]) for i in range(9)]
    for _ in range(4):
        f = _random_state()
        fr = np.zeros(9)
        fr[perm] = f
        g, gr = oracle.collide(f, 1.7), oracle.collide(fr, 1.7)
        expect = np.zeros(9)
        expect[perm] = g
        assert np.allclose(gr, expect, atol=1e-15)
