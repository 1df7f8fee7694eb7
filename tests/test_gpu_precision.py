"""Population storage in FP16 and BF16 (FP32 arithmetic) against the FP64 oracle.

16-bit storage keeps the populations relative to the free-stream equilibrium.  The
bounds below document the precision of each form rather than a target.  On the NACA
0012 small case (alpha 0, Re 1e6, 6 levels, tau - 1/2 ~ 5e-5 on the finest level) the
collision barely damps the shear moments, so the rounding injected at every sub-step
accumulates and the result depends on rounding details: over 300 coarse steps FP16
gave C_D errors between 5e-4 and 4e-3 and BF16 between 9e-3 and 1.4e-2 across builds
that differ only in FP32 rounding (FP32 storage: 1e-4).  The bounds are about twice
the largest error seen.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2601_18443_gb300 as pkg
from paper_2601_18443_gb300 import workloads as W

pytestmark = pytest.mark.gpu
U_LAT = 0.1 * math.sqrt(1.0 / 3.0)

# (store, u rel L2, C_D relative) at 300 coarse steps on the small airfoil case
AIRFOIL_BOUNDS = {1: (1e-3, 1e-2), 2: (1e-2, 3e-2)}
# (store, u rel L2) on the periodic Taylor-Green vortex after 200 steps (the storage shift is
# the free-stream equilibrium, so the zero-mean vortex stores values of order U)
TG_BOUNDS = {1: 2e-3, 2: 4e-2}


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    oracle.build()
    import torch
    torch.cuda.set_device(0)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("store", [1, 2])
def test_taylor_green_16bit_storage(store):
    n = 64
    cfg = W.base_config(levels=1, nx0=n, ny0=n, h0=1.0, Re=U_LAT / 0.05, periodic=1, solid_walls=0,
                        turbulence=0, wall_model=3)
    r = oracle.Solver(cfg)
    r.set_geometry([])
    g = pkg.Solver(dict(cfg, store=store))
    g.set_geometry([])
    k = 2 * np.pi / n
    x = np.arange(n) + 0.5
    X, Y = np.meshgrid(x, x)
    ux, uy = 0.03 * np.sin(k * X) * np.cos(k * Y), -0.03 * np.cos(k * X) * np.sin(k * Y)
    for s in (g, r):
        s.set_fields(0, rho=np.ones_like(X), ux=ux, uy=uy)
    g.step(200); r.step(200)
    a, b = g.get_fields(0), r.get_fields(0)
    e = _rel(np.concatenate([a["ux"].ravel(), a["uy"].ravel()]), np.concatenate([b["ux"].ravel(), b["uy"].ravel()]))
    print("store", store, "u rel L2", e)
    assert e <= TG_BOUNDS[store]


@pytest.mark.parametrize("store", [1, 2])
def test_airfoil_16bit_storage_errors(store):
    cfg, loops = W.naca0012_small()
    r = oracle.Solver(cfg)
    r.set_geometry(loops)
    g = pkg.Solver(dict(cfg, store=store))
    g.set_geometry(loops)
    g.step(300); r.step(300)
    num = den = 0.0
    for l in range(cfg["levels"]):
        a, b = g.get_fields(l), r.get_fields(l)
        act = (b["mask"] == 1) | (b["mask"] == 2)
        num += np.sum((a["ux"] - b["ux"])[act] ** 2 + (a["uy"] - b["uy"])[act] ** 2)
        den += np.sum(b["ux"][act] ** 2 + b["uy"][act] ** 2)
    eu = math.sqrt(num / den)
    lg, lr = g.get_loads(), r.get_loads()
    ecd = abs(lg["CD"] - lr["CD"]) / abs(lr["CD"])
    ecl = abs(lg["CL"] - lr["CL"]) / abs(lr["CD"])
    ecp = _rel(lg["cp"], lr["cp"])
    ecf = _rel(lg["cf"], lr["cf"])
    print(f"store {store}: u {eu:.2e} CD {ecd:.2e} CL/CD {ecl:.2e} Cp {ecp:.2e} Cf {ecf:.2e}")
    bu, bcd = AIRFOIL_BOUNDS[store]
    assert eu <= bu and ecd <= bcd
