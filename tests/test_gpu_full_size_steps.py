"""Parity at the full size of the benchmark workload (NACA 0012 at alpha 10 deg, 6 levels to
c/4096, 1.52M nodes), one launch at a time, against the FP64 oracle's building blocks fed
the GPU's own state before the launch:

- wall records (Sec 2.3 steps 1-5, eq 28): rho_W, u_W, u_tau, chi_B of sampled boundary
  nodes from the finest level's fields;
- one finest-level step: the post-collision populations of sampled boundary nodes, whose
  cut links take Yu's interpolated bounce-back (eq 27, eq 24 fallback) with the wall state,
  then the central-moment collision (eqs 5-10) relaxing with chi_B (Sec 2.2);
- two level pairs (levels 4/5 and 3/4): what the ghost children relay in the fine level's
  odd sub-step (equal to the fine state they pull from, or the parent's exploded value where
  they keep their own), the coarse band cells' step with coalescence (the mean of the four
  children's relays), SA-neg (eqs 12-17) and collision, and the explosion of the result
  into the ghosts (Rohde transfers, Sec 2.1).

The launches are replayed one by one with lbm_step_launch from a checkpoint of a developed
state; every test restores the checkpoint first.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2601_18443_gb300 as pkg
from paper_2601_18443_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CX = np.array([0, 1, -1, 0, 0, 1, -1, 1, -1])
CY = np.array([0, 0, 0, 1, -1, 1, -1, -1, 1])
OPP = np.array([0, 2, 1, 4, 3, 6, 5, 8, 7])
TOL_WALL = 1e-5          # relative L2 over the sampled records, per wall-state column
TOL_POP = 2e-6           # max abs difference of post-collision populations (values near 0.1)
N_SAMPLE = 600


@pytest.fixture(scope="module")
def case():
    import torch

    pkg.build()
    oracle.build()
    torch.cuda.set_device(0)
    cfg, loops = W.naca0012_large()
    g = pkg.Solver(cfg)
    g.set_geometry(loops)
    g.step(3)
    blob = g.get_state()
    yield cfg, g, blob
    g.close()


def _nu(cfg, level):
    U = cfg["Ma"] * math.sqrt(1.0 / 3.0)
    return U * (cfg["chord"] / cfg["h0"]) * 2**level / cfg["Re"]


def _omega(chi, nu):
    c3 = max(chi, 0.0) ** 3
    nut = max(chi, 0.0) * nu * c3 / (c3 + 7.1**3)
    return 1.0 / (3.0 * (nu + nut) + 0.5)


def _at(arr, box, i, j):
    """value of a level array (..., ny, nx) at global cell (i, j)"""
    return arr[..., j - box[1], i - box[0]]


def _wall_expected(cfg, g, F, box, recs):
    ij, geo, nst = g.wall_records()
    sij, _, _ = g.wall_stencils()
    nu = _nu(cfg, cfg["levels"] - 1)
    out = {}
    for r in recs:
        ns = nst[r]
        si, sj = sij[r, :ns, 0], sij[r, :ns, 1]
        dx, dy = si + 0.5 - geo[r, 5], sj + 0.5 - geo[r, 6]
        vals = [_at(F[k], box, si, sj) for k in ("rho", "ux", "uy")]
        out[r] = oracle.wall_point(cfg, nu, dx, dy, *vals, geo[r, 2:4], geo[r, 4])
    return out


def test_wall_records_at_full_size(case):
    cfg, g, blob = case
    g.set_state(blob)
    L = cfg["levels"]
    F = g.get_fields(L - 1)
    box = g.level_box(L - 1)
    st = g.wall_state()
    rng = np.random.default_rng(20261204)
    recs = rng.choice(len(st), size=min(N_SAMPLE, len(st)), replace=False)
    exp = _wall_expected(cfg, g, F, box, recs)
    want = np.array([exp[r] for r in recs])
    got = st[recs]
    for col, name in enumerate(["rhoW", "uWx", "uWy", "utau", "chiB", "tx", "ty", "ut"]):
        e = np.linalg.norm(got[:, col] - want[:, col]) / np.linalg.norm(want[:, col])
        print(name, f"{e:.2e}")
        assert e <= TOL_WALL, (name, e)
    assert np.median(want[:, 3] * 2.0 / _nu(cfg, L - 1)) > 1.0      # y+ at R well away from zero


def test_boundary_nodes_one_finest_step_at_full_size(case):
    cfg, g, blob = case
    g.set_state(blob)
    L = cfg["levels"]
    f = L - 1
    box = g.level_box(f)
    F0, pop0 = g.get_fields(f), g.get_populations(f)
    m = F0["mask"]
    ij, _, _ = g.wall_records()
    ijd, qf = g.cut_links()
    cut = {}
    for (i, j, d), q in zip(ijd, qf):
        cut[(i, j, d)] = q
    rng = np.random.default_rng(7)
    recs = rng.choice(len(ij), size=min(N_SAMPLE, len(ij)), replace=False)
    exp_w = _wall_expected(cfg, g, F0, box, recs)
    g.step_launch(f, 0)                                    # one finest sub-step (even)
    pop1, F1 = g.get_populations(f), g.get_fields(f)
    nu = _nu(cfg, f)
    errs, n_cut, n_half = [], 0, 0
    for r in recs:
        i, j = ij[r]
        w = exp_w[r]
        gpre = np.zeros(9)
        ok = True
        for q in range(9):
            if (i, j, q) in cut:
                qo = OPP[q]
                ni, nj = i + CX[q], j + CY[q]
                nxt = _at(m, box, ni, nj) in (1, 2)
                gpre[q] = oracle.yu_link(q, cut[(i, j, q)], w[0], w[1], w[2],
                                         _at(pop0[qo], box, ni, nj) if nxt else 0.0,
                                         _at(pop0[qo], box, i, j), _at(pop0[q], box, i, j), nxt)
                n_cut += 1
                n_half += not nxt
            else:
                ui, uj = i - CX[q], j - CY[q]
                if _at(m, box, ui, uj) not in (1, 2):
                    ok = False
                gpre[q] = _at(pop0[q], box, ui, uj)
        if not ok:
            continue
        post = oracle.collide(gpre, _omega(w[4], nu), 1.0)
        errs.append(np.abs(_at(pop1, box, i, j) - post).max())
        assert abs(_at(F1["chi"], box, i, j) - w[4]) <= 1e-5 * max(abs(w[4]), 1.0)
    print(f"{len(errs)} boundary nodes, {n_cut} cut links ({n_half} half-way), max population error {max(errs):.2e}")
    assert len(errs) >= 500 and n_cut >= 500
    assert max(errs) <= TOL_POP


def _advance(g, l, restrict, L, hook=None):
    """the recursive level step of Sec 2.1 as single launches; hook(name, level) runs
    before the level's own launch"""
    if l < L - 1:
        g.step_launch(l, 2)
        _advance(g, l + 1, 0, L, hook)
        _advance(g, l + 1, 1, L, hook)
    if hook:
        hook(l)
    g.step_launch(l, 1 if (restrict and l > 0) else 0)


@pytest.mark.parametrize("coarse", [4, 3])
def test_level_pair_relay_coalescence_explosion_at_full_size(case, coarse):
    cfg, g, blob = case
    g.set_state(blob)
    L = cfg["levels"]
    c, fl = coarse, coarse + 1
    snap = {}

    def hook(l):
        # before the fine level's second (odd) sub-step: its state after the even one
        if l == fl and "fineC" not in snap and snap.get("fine_seen", 0) == 1:
            snap["fineC"] = g.get_populations(fl)
        if l == fl:
            snap["fine_seen"] = snap.get("fine_seen", 0) + 1
        if l == c:
            snap["relay"] = g.ghost_relay(c)
            snap["Fc"], snap["popc"] = g.get_fields(c), g.get_populations(c)

    # one step of the coarse level: prolongation, two fine sub-steps, then its own launch
    g.step_launch(c, 2)
    _advance(g, fl, 0, L, hook)
    _advance(g, fl, 1, L, hook)
    hook(c)
    g.step_launch(c, 0)
    popc1, popf1 = g.get_populations(c), g.get_populations(fl)
    boxc, boxf = g.level_box(c), g.level_box(fl)
    flags_f, flags_c = g.flags(fl).astype(np.int64), g.flags(c).astype(np.int64)
    mf = g.mask(fl)
    fineC, popc, Fc = snap["fineC"], snap["popc"], snap["Fc"]
    bij, relay = snap["relay"]
    dc = g.wall_distance(c)
    nu = _nu(cfg, c)
    # band cells inside the section are solid (far from the wall, beside covered cells) and
    # take no step: sample the fluid ones
    mc = g.mask(c)
    fluid = np.nonzero(_at(mc, boxc, bij[:, 0], bij[:, 1]) == 1)[0]
    rng = np.random.default_rng(100 + coarse)
    sel = rng.choice(fluid, size=min(N_SAMPLE, len(fluid)), replace=False)
    n_coal, n_keep, errs = 0, 0, []
    for b in sel:
        i, j = bij[b]
        # (i) relay of each child: the pulled value, or the parent's exploded one
        for mm in range(4):
            ci, cj = 2 * i + (mm & 1), 2 * j + (mm >> 1)
            fw = _at(flags_f, boxf, ci, cj)
            child_fluid = _at(mf, boxf, ci, cj) == 4
            for q in range(1, 9):
                keep = (not child_fluid) or (fw >> (13 + q - 1)) & 1
                want = _at(popc[q], boxc, i, j) if keep else _at(fineC[q], boxf, ci - CX[q], cj - CY[q])
                n_keep += bool(keep)
                assert relay[b, mm, q] == want, (b, mm, q, relay[b, mm, q], want)
        # (ii) the band cell's step: coalesced and pulled populations, SA-neg, collision
        fcw = _at(flags_c, boxc, i, j)
        gpre = np.zeros(9)
        for q in range(9):
            if q > 0 and (fcw >> (5 + q - 1)) & 1:
                gpre[q] = 0.25 * relay[b, :, q].sum()
                n_coal += 1
            else:
                gpre[q] = _at(popc[q], boxc, i - CX[q], j - CY[q])
        st = [np.array([_at(Fc[k], boxc, i + CX[q], j + CY[q]) for q in range(9)]) for k in ("chi", "ux", "uy")]
        chi_new = oracle.sa_update_point(*st, max(_at(dc, boxc, i, j), 0.5), nu, cfg.get("sa_convection", 0))
        post = oracle.collide(gpre, _omega(chi_new, nu), 1.0)
        errs.append(np.abs(_at(popc1, boxc, i, j) - post).max())
        # (iii) explosion: the four ghost children relay the new post-collision populations next
        for mm in range(4):
            ci, cj = 2 * i + (mm & 1), 2 * j + (mm >> 1)
            if _at(mf, boxf, ci, cj) == 4:
                assert np.array_equal(_at(popf1, boxf, ci, cj), _at(popc1, boxc, i, j))
    print(f"levels {c}/{fl}: {len(errs)} band cells, {n_coal} coalesced populations, {n_keep} kept, "
          f"max population error {max(errs):.2e}")
    assert len(errs) >= 500 and n_coal >= 500
    assert max(errs) <= TOL_POP
