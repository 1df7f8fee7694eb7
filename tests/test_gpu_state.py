"""Checkpoint and resume through the C ABI: a solve restored from lbm_get_state, into a new
solver or into the same one (rewind), continues bit for bit; blobs from another grid,
storage precision or set of physical parameters are rejected."""
import numpy as np
import pytest

import paper_2601_18443_gb300 as pkg
from paper_2601_18443_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _pops(s, L):
    return [s.get_populations(l) for l in range(L)]


@pytest.mark.parametrize("store", [0, 1])
def test_resume_continues_bit_for_bit(store):
    pkg.build()
    cfg, loops = W.naca0012_small(levels=5)
    cfg = dict(cfg, store=store)
    L = cfg["levels"]
    a = pkg.Solver(cfg)
    a.set_geometry(loops)
    a.step(7)                                  # odd level-0 parity at the checkpoint
    a.coefficients()
    blob = a.get_state()
    a.step(12)
    want, la = _pops(a, L), a.coefficients()

    b = pkg.Solver(cfg)                        # fresh solver: even parity, other buffers
    b.set_geometry(loops)
    b.set_state(blob)
    assert b.coefficients()["step"] == 7
    b.step(12)
    for l, (x, y) in enumerate(zip(want, _pops(b, L))):
        assert np.array_equal(x, y, equal_nan=True), l
    lb = b.coefficients()
    assert lb["step"] == la["step"] == 19 and abs(lb["CL"] - la["CL"]) < 1e-12

    a.set_state(blob)                          # rewind the same solver
    a.step(12)
    for l, (x, y) in enumerate(zip(want, _pops(a, L))):
        assert np.array_equal(x, y, equal_nan=True), l


def test_state_from_another_grid_is_rejected():
    pkg.build()
    cfg, loops = W.naca0012_small(levels=5)
    a = pkg.Solver(cfg)
    a.set_geometry(loops)
    blob = a.get_state()
    c = pkg.Solver(cfg)
    c.set_geometry([W.naca_loop("0015", cfg["h0"] / 16, alpha_deg=2.0)])
    with pytest.raises(pkg.LBMError) as e:
        c.set_state(blob)
    assert e.value.code == -1
    with pytest.raises(pkg.LBMError):
        a.set_state(blob[:-4])                 # truncated
    d = pkg.Solver(dict(cfg, store=1))
    d.set_geometry(loops)
    with pytest.raises(pkg.LBMError):
        d.set_state(blob)                      # other storage precision


@pytest.mark.parametrize("change", [dict(Re=2.0e6), dict(Ma=0.12), dict(chi_inf=4.0), dict(outlet=0),
                                    dict(sa_convection=1), dict(d_wv=0.9)])
def test_state_from_other_physical_parameters_is_rejected(change):
    # the same grid (identical flag words) but another Reynolds or Mach number, inlet
    # nu_tilde, outlet form, SA convection or virtual-node distance: the blob is refused
    pkg.build()
    cfg, loops = W.naca0012_small(levels=4)
    a = pkg.Solver(cfg)
    a.set_geometry(loops)
    a.step(2)
    blob = a.get_state()
    b = pkg.Solver(dict(cfg, **change))
    b.set_geometry(loops)
    with pytest.raises(pkg.LBMError) as e:
        b.set_state(blob)
    assert e.value.code == -1
    a.set_state(blob)                          # the same configuration still accepts it
