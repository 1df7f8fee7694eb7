"""FP64 CPU oracle of the LBM-RANS step (Ponsin & Lozano, arXiv 2601.18443).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library never loads it and shares no code with it.

The C source (``oracle.c``) is compiled with gcc into ``_build/liboracle.so`` on
first use (or by ``build()``) and driven through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (-O2, OpenMP, no FMA contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off", "-std=gnu11",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Config(C.Structure):
    _fields_ = [
        ("levels", C.c_int), ("nx0", C.c_int), ("ny0", C.c_int),
        ("x0", C.c_double), ("y0", C.c_double), ("h0", C.c_double),
        ("layers", C.c_int),
        ("chord", C.c_double), ("Re", C.c_double), ("Ma", C.c_double),
        ("chi_inf", C.c_double), ("d_wr", C.c_double), ("d_wv", C.c_double),
        ("turbulence", C.c_int), ("wall_model", C.c_int), ("periodic", C.c_int),
        ("solid_walls", C.c_int), ("sa_convection", C.c_int), ("outlet", C.c_int),
    ]


class Loads(C.Structure):
    _fields_ = [("CL", C.c_double), ("CD", C.c_double), ("CDp", C.c_double), ("CDf", C.c_double),
                ("mass", C.c_double), ("dCL", C.c_double), ("step", C.c_longlong)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            L.oracle_create.argtypes = [C.POINTER(Config), C.POINTER(C.c_void_p)]
            L.oracle_destroy.argtypes = [C.c_void_p]
            L.oracle_set_threads.argtypes = [C.c_int]
            L.oracle_set_threads.restype = None
            L.oracle_last_error.argtypes = [C.c_void_p]
            L.oracle_last_error.restype = C.c_char_p
            L.oracle_set_geometry.argtypes = [C.c_void_p, dp, ip, C.c_int]
            L.oracle_set_wall_slip.argtypes = [C.c_void_p, dp, C.c_int]
            L.oracle_step.argtypes = [C.c_void_p, C.c_int]
            L.oracle_level_box.argtypes = [C.c_void_p, C.c_int, ip, ip, ip, ip]
            L.oracle_get_fields.argtypes = [C.c_void_p, C.c_int, dp, dp, dp, dp, C.c_void_p, C.c_int]
            L.oracle_set_fields.argtypes = [C.c_void_p, C.c_int, dp, dp, dp, dp]
            L.oracle_get_loads.argtypes = [C.c_void_p, C.POINTER(Loads), dp, dp, C.c_int, ip]
            L.oracle_get_cut_links.argtypes = [C.c_void_p, ip, dp, C.c_int, ip]
            L.oracle_get_wall_records.argtypes = [C.c_void_p, ip, dp, ip, C.c_int, ip]
            L.oracle_get_wall_state.argtypes = [C.c_void_p, dp, C.c_int, ip]
            L.oracle_get_wall_distance.argtypes = [C.c_void_p, C.c_int, dp, C.c_int]
            L.oracle_set_walls.argtypes = [C.c_void_p, dp, ip, C.c_int]
            L.oracle_probe_cells.argtypes = [C.c_void_p, C.c_int, ip, C.c_int, C.c_void_p, C.c_void_p, dp]
            L.oracle_probe_links.argtypes = [C.c_void_p, ip, C.c_int, dp]
            L.oracle_mass.argtypes = [C.c_void_p]
            L.oracle_mass.restype = C.c_double
            L.oracle_wf_uplus.argtypes = [C.c_double]
            L.oracle_wf_uplus.restype = C.c_double
            L.oracle_wf_dudy.argtypes = [C.c_double]
            L.oracle_wf_dudy.restype = C.c_double
            L.oracle_wf_utau.argtypes = [C.c_double, C.c_double, C.c_double]
            L.oracle_wf_utau.restype = C.c_double
            L.oracle_feq.argtypes = [C.c_double, C.c_double, C.c_double, dp]
            L.oracle_collide.argtypes = [dp, C.c_double, C.c_double, dp]
            L.oracle_sa_source.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, dp, dp]
            L.oracle_sa_update_point.argtypes = [dp, dp, dp, C.c_double, C.c_double, C.c_int]
            L.oracle_sa_convection.argtypes = [dp, C.c_double, C.c_double, C.c_int]
            L.oracle_wall_point.argtypes = [C.POINTER(Config), C.c_double, C.c_int, dp, dp, dp, dp, dp, dp, C.c_double,
                                            dp, dp]
            L.oracle_wall_point.restype = None
            L.oracle_yu_link.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                         C.c_double, C.c_double, C.c_int]
            L.oracle_yu_link.restype = C.c_double
            L.oracle_sa_convection.restype = C.c_double
            L.oracle_sa_update_point.restype = C.c_double
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


# --- building blocks -------------------------------------------------------

def wf_uplus(yp):
    return lib().oracle_wf_uplus(float(yp))


def wf_dudy(yp):
    return lib().oracle_wf_dudy(float(yp))


def wf_utau(ut, y, nu):
    return lib().oracle_wf_utau(float(ut), float(y), float(nu))


def feq(rho, ux, uy):
    out = np.zeros(9)
    lib().oracle_feq(rho, ux, uy, _dp(out))
    return out


def collide(f, omega_nu, omega_b=1.0):
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(9)
    lib().oracle_collide(_dp(f), omega_nu, omega_b, _dp(out))
    return out


def sa_source(chi, nu, vort, d):
    P = np.zeros(1)
    D = np.zeros(1)
    lib().oracle_sa_source(chi, nu, vort, d, _dp(P), _dp(D))
    return float(P[0]), float(D[0])


def sa_update_point(chi9, ux9, uy9, d, nu, convection=0):
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (chi9, ux9, uy9)]
    return lib().oracle_sa_update_point(_dp(a[0]), _dp(a[1]), _dp(a[2]), d, nu, int(convection))


def sa_convection(nt9, u, v, scheme=0):
    a = np.ascontiguousarray(nt9, dtype=np.float64)
    return lib().oracle_sa_convection(_dp(a), float(u), float(v), int(scheme))


def wall_point(cfg, nu, dx, dy, rho, ux, uy, n, dwb, slip=(0.0, 0.0)):
    """Wall state of one boundary node from its stencil (Sec 2.3 steps 1-5): rho_W, u_W
    (2), u_tau, chi_B, t (2), |u_Rt|; dx, dy: stencil cell centres relative to R."""
    c = Config()
    for name, _ in Config._fields_:
        setattr(c, name, cfg.get(name, 0))
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (dx, dy, rho, ux, uy, n, slip)]
    out = np.zeros(8)
    lib().oracle_wall_point(C.byref(c), float(nu), len(a[0]), *[_dp(x) for x in a[:6]], float(dwb), _dp(a[6]), _dp(out))
    return out


def yu_link(q, qf, rhoW, uWx, uWy, f_qo_next, f_qo_B, f_q_B, next_fluid):
    """Yu's interpolated slip bounce-back for pulled direction q (eq 27, eq 24 fallback)."""
    return lib().oracle_yu_link(int(q), float(qf), float(rhoW), float(uWx), float(uWy), float(f_qo_next),
                                float(f_qo_B), float(f_q_B), int(bool(next_fluid)))


# --- solver ------------------------------------------------------------------

class OracleError(RuntimeError):
    pass


class Solver:
    """FP64 reference solver; same call shapes as the product's C ABI."""

    def __init__(self, cfg: dict):
        self._lib = lib()
        c = Config()
        for name, _ in Config._fields_:
            setattr(c, name, cfg.get(name, 0))
        self.cfg = dict(cfg)
        h = C.c_void_p()
        rc = self._lib.oracle_create(C.byref(c), C.byref(h))
        if rc != 0:
            raise OracleError(f"oracle_create failed ({rc})")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _check(self, rc):
        if rc != 0:
            raise OracleError(f"{rc}: {self._lib.oracle_last_error(self._h).decode()}")

    def set_geometry(self, loops):
        """loops: list of (n, 2) arrays of closed polylines (first vertex not repeated)."""
        xy = np.ascontiguousarray(np.concatenate([np.asarray(p, dtype=np.float64) for p in loops])
                                  if loops else np.zeros((0, 2)))
        off = np.zeros(len(loops) + 1, dtype=np.int32)
        off[1:] = np.cumsum([len(p) for p in loops])
        self._check(self._lib.oracle_set_geometry(self._h, _dp(xy), _ip(off), len(loops)))
        self.n_loops = len(loops)

    def set_walls(self, loops):
        """Snap the wall polylines without building the levels (for the point probes)."""
        xy = np.ascontiguousarray(np.concatenate([np.asarray(p, dtype=np.float64) for p in loops])
                                  if loops else np.zeros((0, 2)))
        off = np.zeros(len(loops) + 1, dtype=np.int32)
        off[1:] = np.cumsum([len(p) for p in loops])
        self._check(self._lib.oracle_set_walls(self._h, _dp(xy), _ip(off), len(loops)))

    def probe_cells(self, level, ij):
        """solid flag, refinement test of level + 1, and wall distance of level cells ij (n, 2)."""
        ij = np.ascontiguousarray(ij, dtype=np.int32)
        n = len(ij)
        solid = np.zeros(n, dtype=np.uint8)
        near = np.zeros(n, dtype=np.uint8)
        dist = np.zeros(n)
        self._check(self._lib.oracle_probe_cells(self._h, level, _ip(ij), n, solid.ctypes.data_as(C.c_void_p),
                                                 near.ctypes.data_as(C.c_void_p), _dp(dist)))
        return solid, near, dist

    def probe_links(self, ijd):
        """wall fraction q of finest-level links ijd (n, 3) = (i, j, pulled direction)."""
        ijd = np.ascontiguousarray(ijd, dtype=np.int32)
        q = np.zeros(len(ijd))
        self._check(self._lib.oracle_probe_links(self._h, _ip(ijd), len(ijd), _dp(q)))
        return q

    def set_wall_slip(self, uw):
        uw = np.ascontiguousarray(uw, dtype=np.float64).reshape(-1)
        self._check(self._lib.oracle_set_wall_slip(self._h, _dp(uw), len(uw) // 2))

    def step(self, n=1):
        self._check(self._lib.oracle_step(self._h, int(n)))

    def level_box(self, level):
        v = [C.c_int() for _ in range(4)]
        self._check(self._lib.oracle_level_box(self._h, level, *[C.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def get_fields(self, level):
        i0, j0, nx, ny = self.level_box(level)
        rho, ux, uy, chi = (np.zeros((ny, nx)) for _ in range(4))
        mask = np.zeros((ny, nx), dtype=np.uint8)
        self._check(self._lib.oracle_get_fields(self._h, level, _dp(rho), _dp(ux), _dp(uy), _dp(chi),
                                                mask.ctypes.data_as(C.c_void_p), nx * ny))
        return dict(rho=rho, ux=ux, uy=uy, chi=chi, mask=mask, i0=i0, j0=j0)

    def set_fields(self, level, rho=None, ux=None, uy=None, chi=None):
        i0, j0, nx, ny = self.level_box(level)
        arrs = []
        for a in (rho, ux, uy, chi):
            arrs.append(None if a is None else np.ascontiguousarray(np.broadcast_to(a, (ny, nx)), dtype=np.float64))
        ptrs = [None if a is None else _dp(a) for a in arrs]
        self._check(self._lib.oracle_set_fields(self._h, level, *ptrs))

    def get_loads(self):
        out = Loads()
        n = C.c_int()
        self._check(self._lib.oracle_get_loads(self._h, C.byref(out), None, None, 0, C.byref(n)))
        cap = n.value
        cp = np.zeros(max(cap, 1))
        cf = np.zeros(max(cap, 1))
        self._check(self._lib.oracle_get_loads(self._h, C.byref(out), _dp(cp), _dp(cf), cap, C.byref(n)))
        d = {k: getattr(out, k) for k, _ in Loads._fields_}
        d["cp"] = cp[:cap]
        d["cf"] = cf[:cap]
        return d

    def mass(self):
        return self._lib.oracle_mass(self._h)

    def cut_links(self):
        n = C.c_int()
        self._lib.oracle_get_cut_links(self._h, None, None, 0, C.byref(n))
        ijd = np.zeros((max(n.value, 1), 3), dtype=np.int32)
        q = np.zeros(max(n.value, 1))
        self._check(self._lib.oracle_get_cut_links(self._h, _ip(ijd), _dp(q), n.value, C.byref(n)))
        return ijd[:n.value], q[:n.value]

    def wall_records(self):
        n = C.c_int()
        self._lib.oracle_get_wall_records(self._h, None, None, None, 0, C.byref(n))
        m = max(n.value, 1)
        ij = np.zeros((m, 2), dtype=np.int32)
        geo = np.zeros((m, 9))
        ns = np.zeros(m, dtype=np.int32)
        self._check(self._lib.oracle_get_wall_records(self._h, _ip(ij), _dp(geo), _ip(ns), n.value, C.byref(n)))
        return ij[:n.value], geo[:n.value], ns[:n.value]

    def wall_state(self):
        n = C.c_int()
        self._lib.oracle_get_wall_state(self._h, None, 0, C.byref(n))
        st = np.zeros((max(n.value, 1), 8))
        self._check(self._lib.oracle_get_wall_state(self._h, _dp(st), n.value, C.byref(n)))
        return st[:n.value]

    def wall_distance(self, level):
        i0, j0, nx, ny = self.level_box(level)
        d = np.zeros((ny, nx))
        self._check(self._lib.oracle_get_wall_distance(self._h, level, _dp(d), nx * ny))
        return d


def threads() -> int:
    return lib().oracle_threads()


def set_threads(n: int) -> None:
    """OpenMP team size of the oracle's parallel regions started from this thread."""
    lib().oracle_set_threads(int(n))
