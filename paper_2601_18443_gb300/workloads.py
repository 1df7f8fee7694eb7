"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method: it only generates wall polylines
(analytic NACA 4-digit sections, rectangles, channels) and the solver
configurations of the workloads.  Both the CUDA library and the CPU oracle
receive the same arrays from here.

The paper's own geometries (the NASA TMR NACA 0012 coordinates and the HLPW
MD-30P30N) are not available; analytic NACA sections stand in for them.
"""
from __future__ import annotations

import math

import numpy as np


def naca4(m: float, p: float, t: float, n: int) -> np.ndarray:
    """Closed NACA 4-digit section of unit chord, leading edge at the origin.

    Standard analytic thickness and mean-line formulas with the closed
    trailing-edge coefficient; cosine spacing with ``n`` intervals per surface.
    The loop runs trailing edge -> upper surface -> leading edge -> lower
    surface (counter-clockwise); the first vertex is not repeated.
    """
    beta = np.linspace(math.pi, 0.0, n + 1)
    x = 0.5 * (1.0 - np.cos(beta))                      # 1 -> 0
    yt = np.maximum(5.0 * t * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x**2 + 0.2843 * x**3 - 0.1036 * x**4), 0.0)
    if m > 0.0 and p > 0.0:
        yc = np.where(x < p, m / p**2 * (2 * p * x - x**2), m / (1 - p)**2 * ((1 - 2 * p) + 2 * p * x - x**2))
        dyc = np.where(x < p, 2 * m / p**2 * (p - x), 2 * m / (1 - p)**2 * (p - x))
    else:
        yc = np.zeros_like(x)
        dyc = np.zeros_like(x)
    th = np.arctan(dyc)
    xu, yu = x - yt * np.sin(th), yc + yt * np.cos(th)
    xl, yl = x + yt * np.sin(th), yc - yt * np.cos(th)
    upper = np.stack([xu, yu], axis=1)                  # TE .. LE (n+1 points)
    lower = np.stack([xl, yl], axis=1)[::-1][1:-1]      # after LE .. before TE
    return np.concatenate([upper, lower], axis=0)


def transform(loop: np.ndarray, chord=1.0, alpha_deg=0.0, pivot=(0.25, 0.0), offset=(0.0, 0.0)) -> np.ndarray:
    """Scale by chord, rotate nose-up by alpha about the pivot (freestream +x), translate."""
    a = -math.radians(alpha_deg)
    R = np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])
    pv = np.asarray(pivot, dtype=np.float64) * chord
    out = (loop * chord - pv) @ R.T + pv
    return out + np.asarray(offset, dtype=np.float64)


def naca_loop(code: str, h_finest: float, chord=1.0, alpha_deg=0.0, pivot=(0.25, 0.0), offset=(0.0, 0.0),
              max_seg_frac=0.5) -> np.ndarray:
    """NACA section with every segment shorter than max_seg_frac * h_finest."""
    m, p, t = int(code[0]) / 100.0, int(code[1]) / 10.0, int(code[2:]) / 100.0
    n = max(16, int(math.ceil(math.pi * chord / (max_seg_frac * h_finest))))
    while True:
        loop = naca4(m, p, t, n)
        seg = np.linalg.norm(np.diff(np.vstack([loop, loop[:1]]), axis=0), axis=1) * chord
        if seg.max() <= max_seg_frac * h_finest:
            break
        n = int(n * 1.25) + 1
    return transform(loop, chord, alpha_deg, pivot, offset)


def rectangle(x0, y0, x1, y1) -> np.ndarray:
    return np.array([[x0, y0], [x1, y0], [x1, y1], [x0, y1]], dtype=np.float64)


def l_shape(x0, y0, x1, y1, xm, ym) -> np.ndarray:
    """L-shaped loop: the rectangle [x0,x1]x[y0,y1] minus the corner (xm,x1]x(ym,y1]."""
    return np.array([[x0, y0], [x1, y0], [x1, ym], [xm, ym], [xm, y1], [x0, y1]], dtype=np.float64)


def base_config(**kw) -> dict:
    cfg = dict(levels=1, nx0=64, ny0=64, x0=0.0, y0=0.0, h0=1.0, layers=8, chord=1.0, Re=1000.0, Ma=0.1,
               chi_inf=3.0, d_wr=2.0, d_wv=1.0, turbulence=0, wall_model=3, periodic=0, solid_walls=1,
               sa_convection=0, outlet=1)
    cfg.update(kw)
    return cfg


# --- named workloads ----------------------------------------------------------

def naca0012_small(levels=6):
    """NACA 0012, alpha 0, Re 1e6, Ma 0.1; coarse 128 x 64 over a 16c x 8c box
    (h0 = c/8), six 2:1 levels to h = c/256; SA-neg with nu_t~ = 3 nu."""
    h0 = 1.0 / 8.0
    cfg = base_config(levels=levels, nx0=128, ny0=64, x0=-5.5, y0=-4.0, h0=h0, layers=8, chord=1.0, Re=1.0e6,
                      Ma=0.1, turbulence=1, wall_model=0, periodic=0, solid_walls=1)
    hf = h0 / 2 ** (levels - 1)
    return cfg, [naca_loop("0012", hf, alpha_deg=0.0)]


def naca0012_large(box=(8.0, 4.0), layers=56):
    """NACA 0012, alpha 10 deg, Re 6e6, Ma 0.15; six 2:1 levels with the finest
    spacing c/4096 (h0 = c/128) over an 8c x 4c box; 56 cells per refinement band
    give 1.52M active nodes and 21.4M node updates per coarse step."""
    h0 = 1.0 / 128.0
    nx0, ny0 = int(round(box[0] / h0)), int(round(box[1] / h0))
    cfg = base_config(levels=6, nx0=nx0, ny0=ny0, x0=-0.375 * box[0] + 0.25, y0=-0.5 * box[1], h0=h0,
                      layers=layers, chord=1.0, Re=6.0e6, Ma=0.15, turbulence=1, wall_model=0, periodic=0,
                      solid_walls=1)
    hf = h0 / 32.0
    return cfg, [naca_loop("0012", hf, alpha_deg=10.0)]


def noise_field(shape, amplitude, seed):
    """Seeded uniform noise in [-amplitude, amplitude]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-amplitude, amplitude, size=shape)


def highlift_loops(h_finest, alpha_deg=8.0, gap=0.02, overlap=0.02):
    """Synthetic three-element high-lift section (chord c = 1 of the main element):
    slat NACA 2412 of chord 0.15 deflected 30 deg nose-down, main NACA 4412, flap NACA
    2412 of chord 0.3 deflected 30 deg trailing-edge-down, the whole set rotated to
    alpha about the main element's quarter chord.

    Placement: the slat trailing edge sits `overlap` aft of the main leading edge and
    `gap` above the main upper surface there; the flap leading edge sits `overlap` ahead
    of the main trailing edge and `gap` below the main trailing edge plus the flap's
    own half-thickness near its nose (so that the slot is about `gap` wide)."""
    main = naca_loop("4412", h_finest)
    # slat: rotate about its own trailing edge, then move that edge to its station
    slat = naca_loop("2412", h_finest / 0.15, chord=1.0) * 0.15
    slat = transform(slat, 1.0, -30.0, pivot=(slat[0, 0], slat[0, 1]))
    xs = overlap
    m, p, t = 0.04, 0.4, 0.12
    yt = 5 * t * (0.2969 * xs**0.5 - 0.1260 * xs - 0.3516 * xs**2 + 0.2843 * xs**3 - 0.1036 * xs**4)
    yc = m / p**2 * (2 * p * xs - xs**2)
    slat = slat + (np.array([xs, yc + yt + gap]) - slat[0])
    # flap: rotate about its own leading edge, then move that edge to its station
    flap = naca_loop("2412", h_finest / 0.3, chord=1.0) * 0.3
    le = flap[np.argmin(flap[:, 0])]
    flap = transform(flap, 1.0, 30.0, pivot=(le[0], le[1]))
    le = flap[np.argmin(flap[:, 0])]
    half = 0.3 * 0.12 * 0.5
    flap = flap + (np.array([1.0 - overlap, -gap - half]) - le)
    loops = [slat, main, flap]
    return [transform(lp, 1.0, alpha_deg) for lp in loops]


def highlift_3element(levels=8, layers=128, box=(16.0, 8.0), h0=1.0 / 64.0):
    """Synthetic three-element high-lift case: alpha 8 deg, Re 9e6, Ma 0.2, SA-neg, the
    virtual-node wall function; `levels` 2:1 levels from h0 (finest h0 / 2^(levels-1)).
    Defaults: 8 levels from c/64 to c/8192 over a 16c x 8c box, 128 cells per band:
    7.46M active nodes, 555M node updates per coarse step."""
    nx0, ny0 = int(round(box[0] / h0)), int(round(box[1] / h0))
    nx0 -= nx0 % 32
    ny0 -= ny0 % 8
    cfg = base_config(levels=levels, nx0=nx0, ny0=ny0, x0=-0.35 * box[0], y0=-0.5 * box[1], h0=h0, layers=layers,
                      chord=1.0, Re=9.0e6, Ma=0.2, turbulence=1, wall_model=0, periodic=0, solid_walls=1)
    hf = h0 / 2 ** (levels - 1)
    return cfg, highlift_loops(hf)


# --- polar-solve requests (serving) ---------------------------------------------

def polar_requests(n=256, seed=2026, rate_per_s=2.0):
    """Seeded polar-solve requests: Poisson arrivals (mean rate_per_s), NACA 4-digit
    sections with m in 0..4, p in 2..5 (tenths), t in 09..18, alpha ~ U[-4, 16] deg,
    Re ~ logU[1e6, 1e7], 4..7 levels; FP16 (shifted) population storage, Ma 0.15."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
    out = []
    for k in range(n):
        m = int(rng.integers(0, 5))
        p = int(rng.integers(2, 6))
        th = int(rng.integers(9, 19))
        code = f"{m}{p if m else 0}{th:02d}"
        out.append(dict(rid=k, arrival=float(t[k]), code=code, alpha=float(rng.uniform(-4.0, 16.0)),
                        Re=float(10.0 ** rng.uniform(6.0, 7.0)), levels=int(rng.integers(4, 8)), Ma=0.15, store=1))
    return out


def polar_case(req, h0=1.0 / 16.0, box=(16.0, 8.0)):
    """Solver configuration and wall loop of one polar request: a 16c x 8c box at c/16 with
    req['levels'] 2:1 levels (finest c/128 .. c/1024); 16..32 cells per refinement band.
    About 4e4..2e5 active cells and 9e4..6.5e6 node updates per level-0 step."""
    levels = req["levels"]
    layers = {4: 16, 5: 24, 6: 32, 7: 32}[levels]
    nx0, ny0 = int(round(box[0] / h0)), int(round(box[1] / h0))
    cfg = base_config(levels=levels, nx0=nx0, ny0=ny0, x0=-0.375 * box[0] + 0.25, y0=-0.5 * box[1], h0=h0,
                      layers=layers, chord=1.0, Re=req["Re"], Ma=req["Ma"], turbulence=1, wall_model=0, periodic=0,
                      solid_walls=1, store=req.get("store", 1))
    hf = h0 / 2 ** (levels - 1)
    return cfg, [naca_loop(req["code"], hf, alpha_deg=req["alpha"])]
