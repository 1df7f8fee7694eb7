"""GB300-native (sm_103a) LBM-RANS hot path of Ponsin & Lozano (arXiv 2601.18443).

Thin ctypes binding over the C ABI in ``include/lbm.h`` (``liblbm.so`` built
in-tree from ``csrc/``).  Argument marshalling only: every step of the path runs
in the library's CUDA kernels.  There is no CPU fallback; if the library is not
built the binding raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build_ext

__all__ = ["Solver", "LBMError", "library", "build"]

_lib = None


class LBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lbm status {code}: {msg}")
        self.code = code


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class lbm_config(C.Structure):
    _fields_ = [
        ("levels", C.c_int), ("nx0", C.c_int), ("ny0", C.c_int),
        ("x0", C.c_double), ("y0", C.c_double), ("h0", C.c_double),
        ("layers", C.c_int),
        ("chord", C.c_double), ("Re", C.c_double), ("Ma", C.c_double),
        ("chi_inf", C.c_double), ("d_wr", C.c_double), ("d_wv", C.c_double),
        ("turbulence", C.c_int), ("wall_model", C.c_int), ("periodic", C.c_int),
        ("solid_walls", C.c_int), ("store", C.c_int), ("sa_convection", C.c_int),
        ("outlet", C.c_int), ("cuda_stream", C.c_void_p),
        ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_ctx", C.c_void_p),
    ]


class lbm_loads(C.Structure):
    _fields_ = [("CL", C.c_double), ("CD", C.c_double), ("CDp", C.c_double), ("CDf", C.c_double),
                ("mass", C.c_double), ("dCL", C.c_double), ("step", C.c_longlong)]


class lbm_info(C.Structure):
    _fields_ = [("levels", C.c_int), ("cells_active", C.c_longlong * 16), ("cells_present", C.c_longlong * 16),
                ("slots", C.c_longlong * 16), ("node_updates_per_step", C.c_longlong),
                ("wall_records", C.c_longlong), ("cut_links", C.c_longlong), ("surface_segments", C.c_longlong),
                ("kernels_per_step", C.c_longlong), ("bytes_per_node_update", C.c_double),
                ("device_bytes", C.c_double), ("work_tiles", C.c_longlong * 16), ("work_warps", C.c_longlong * 16)]


class lbm_plan(C.Structure):
    _fields_ = [("levels", C.c_int), ("cells_active", C.c_longlong * 16), ("node_updates_per_step", C.c_longlong),
                ("wall_records", C.c_longlong), ("device_bytes", C.c_double), ("reason", C.c_char * 128)]


class lbm_kernel_times(C.Structure):
    _fields_ = [("n_classes", C.c_int), ("name", (C.c_char * 32) * 8), ("total_ms", C.c_double * 8),
                ("launches", C.c_longlong * 8), ("cells", C.c_longlong * 8)]


class lbm_load_record(C.Structure):
    _fields_ = [("step", C.c_longlong), ("CL", C.c_double), ("CD", C.c_double), ("CDp", C.c_double),
                ("CDf", C.c_double), ("mass", C.c_double)]


class lbm_launch_time(C.Structure):
    _fields_ = [("graph", C.c_int), ("level", C.c_int), ("kind", C.c_int), ("blocks", C.c_int),
                ("t_wait_us", C.c_double), ("t_end_us", C.c_double)]


TUNE_CANDIDATES = 12
SCHED_TILE, SCHED_PERSIST, SCHED_WARPS, SCHED_WARPS4 = 0, 1, 2, 3   # LBM_SCHED_* of include/lbm.h


class lbm_tune_report(C.Structure):
    _fields_ = [("levels", C.c_int), ("candidate_min_blocks", C.c_int * TUNE_CANDIDATES),
                ("candidate_sched", C.c_int * TUNE_CANDIDATES), ("candidate_shape", C.c_int * TUNE_CANDIDATES),
                ("level_us", (C.c_double * 16) * TUNE_CANDIDATES), ("min_blocks", C.c_int * 16),
                ("sched", C.c_int * 16), ("shape", C.c_int * 16),
                ("step_us_confirm", C.c_double * (3 + TUNE_CANDIDATES)), ("confirm_choice", C.c_int),
                ("default_step_us", C.c_double), ("step_us", C.c_double * 2),
                ("pdl", C.c_int), ("steps_taken", C.c_longlong)]


def build(force: bool = False, verbose: bool = False) -> str:
    return _build_ext.build(force=force, verbose=verbose)


def library():
    """Load liblbm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build_ext.SO):
        raise RuntimeError("liblbm.so is not built: run __graft_entry__.build() (the CUDA library is required)")
    _lib = _load(_build_ext.SO)
    return _lib


_lib_check = None


def checked_library():
    """liblbm_check.so, the bounds-checked build (built on first use): every index the level
    step follows from a table is checked on the device, and one outside its buffer makes the
    next synchronising call fail.  Pass it as Solver(..., library=checked_library())."""
    global _lib_check
    if _lib_check is None:
        _lib_check = _load(_build_ext.build(bounds_check=True))
    return _lib_check


def _load(path):
    L = C.CDLL(path)
    vp, ip, dp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)
    sig = {
        "lbm_create": ([C.POINTER(lbm_config), C.POINTER(vp)], C.c_int),
        "lbm_create_host": ([C.POINTER(lbm_config), C.POINTER(vp)], C.c_int),
        "lbm_set_geometry": ([vp, dp, ip, C.c_int], C.c_int),
        "lbm_set_wall_slip": ([vp, dp, C.c_int], C.c_int),
        "lbm_plan_geometry": ([C.POINTER(lbm_config), dp, ip, C.c_int, C.POINTER(lbm_plan)], C.c_int),
        "lbm_grid_digest": ([C.POINTER(lbm_config), dp, ip, C.c_int, C.POINTER(C.c_ulonglong)], C.c_int),
        "lbm_set_host_threads": ([C.c_int], None),
        "lbm_step": ([vp, C.c_int], C.c_int),
        "lbm_step_async": ([vp, C.c_int], C.c_int),
        "lbm_synchronize": ([vp], C.c_int),
        "lbm_get_level_box": ([vp, C.c_int, ip, ip, ip, ip], C.c_int),
        "lbm_get_fields": ([vp, C.c_int, dp, dp, dp, dp, vp, C.c_int], C.c_int),
        "lbm_set_fields": ([vp, C.c_int, dp, dp, dp, dp], C.c_int),
        "lbm_get_populations": ([vp, C.c_int, dp, C.c_longlong], C.c_int),
        "lbm_step_launch": ([vp, C.c_int, C.c_int], C.c_int),
        "lbm_batch_create": ([C.POINTER(vp), C.c_int, C.POINTER(vp)], C.c_int),
        "lbm_batch_step": ([vp, C.c_int], C.c_int),
        "lbm_batch_info": ([vp, ip, ip, C.POINTER(C.c_longlong)], C.c_int),
        "lbm_batch_last_error": ([vp], C.c_char_p),
        "lbm_batch_destroy": ([vp], None),
        "lbm_get_ghost_relay": ([vp, C.c_int, ip, dp, C.c_int, ip], C.c_int),
        "lbm_get_loads": ([vp, C.POINTER(lbm_loads), dp, dp, C.c_int, ip], C.c_int),
        "lbm_get_cut_links": ([vp, ip, dp, C.c_int, ip], C.c_int),
        "lbm_get_wall_records": ([vp, ip, dp, ip, C.c_int, ip], C.c_int),
        "lbm_get_wall_state": ([vp, dp, C.c_int, ip], C.c_int),
        "lbm_get_wall_stencils": ([vp, ip, dp, dp, C.c_int, ip], C.c_int),
        "lbm_get_segment_map": ([vp, dp, ip, dp, C.c_int, ip], C.c_int),
        "lbm_get_wall_distance": ([vp, C.c_int, dp, C.c_int], C.c_int),
        "lbm_get_flags": ([vp, C.c_int, C.POINTER(C.c_uint), C.c_int], C.c_int),
        "lbm_get_work_list": ([vp, C.c_int, C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_int)], C.c_int),
        "lbm_get_prolong_independence": ([vp, C.POINTER(C.c_int), C.c_int], C.c_int),
        "lbm_get_info": ([vp, C.POINTER(lbm_info)], C.c_int),
        "lbm_time_kernels": ([vp, C.c_int, C.POINTER(lbm_kernel_times)], C.c_int),
        "lbm_autotune": ([vp, C.c_int, C.POINTER(lbm_tune_report)], C.c_int),
        "lbm_set_launch_variant": ([vp, ip, ip, ip, C.c_int], C.c_int),
        "lbm_set_prolong_merge": ([vp, C.c_int, C.POINTER(C.c_int)], C.c_int),
        "lbm_set_timeline": ([vp, C.c_int], C.c_int),
        "lbm_set_load_history": ([vp, C.c_int, C.c_int], C.c_int),
        "lbm_get_load_history": ([vp, C.c_void_p, C.c_int, C.POINTER(C.c_int)], C.c_int),
        "lbm_get_timeline": ([vp, C.c_void_p, C.c_int, C.POINTER(C.c_int)], C.c_int),
        "lbm_get_state": ([vp, vp, C.c_size_t, C.POINTER(C.c_size_t)], C.c_int),
        "lbm_set_state": ([vp, vp, C.c_size_t], C.c_int),
        "lbm_level_mass_noalloc": ([vp, vp, vp, vp, vp, C.c_longlong, C.c_double, vp, vp, vp], C.c_int),
        "lbm_last_error": ([vp], C.c_char_p),
        "lbm_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _config_struct(cfg):
    c = lbm_config()
    for name, _ in lbm_config._fields_:
        if name in ("cuda_stream", "dev_alloc", "dev_free", "alloc_ctx"):
            continue
        setattr(c, name, cfg.get(name, 0))
    return c


def _loops_arrays(loops):
    xy = np.ascontiguousarray(np.concatenate([np.asarray(p, dtype=np.float64) for p in loops])
                              if loops else np.zeros((0, 2)))
    off = np.zeros(len(loops) + 1, dtype=np.int32)
    off[1:] = np.cumsum([len(p) for p in loops])
    return xy, off


def plan(cfg: dict, loops) -> dict:
    """lbm_plan_geometry: device bytes and active cells of a solve, without a GPU."""
    c = _config_struct(cfg)
    xy, off = _loops_arrays(loops)
    out = lbm_plan()
    rc = library().lbm_plan_geometry(C.byref(c), _dp(xy), _ip(off), len(loops), C.byref(out))
    if rc != 0:
        raise LBMError(rc, "lbm_plan_geometry: " + out.reason.decode())
    L = out.levels
    return dict(levels=L, cells_active=list(out.cells_active[:L]), node_updates_per_step=out.node_updates_per_step,
                wall_records=out.wall_records, device_bytes=out.device_bytes)


def set_host_threads(n: int) -> None:
    """lbm_set_host_threads: host threads of the grid builds started from this thread."""
    library().lbm_set_host_threads(int(n))


def grid_digest(cfg: dict, loops) -> int:
    """lbm_grid_digest: 64-bit digest of the host-built grid tables, without a GPU."""
    c = _config_struct(cfg)
    xy, off = _loops_arrays(loops)
    out = C.c_ulonglong(0)
    rc = library().lbm_grid_digest(C.byref(c), _dp(xy), _ip(off), len(loops), C.byref(out))
    if rc != 0:
        raise LBMError(rc, "lbm_grid_digest")
    return int(out.value)


class Solver:
    """One LBM-RANS solve on the current CUDA device (see include/lbm.h).

    host_only=True gives a handle without device state (lbm_create_host): it builds the
    grid tables on the host and answers the table queries (level_box, mask,
    wall_distance, cut_links, wall_records) on machines without a GPU."""

    def __init__(self, cfg: dict, stream=None, torch_allocator: bool = False, host_only: bool = False,
                 library=None):
        self._lib = library if library is not None else globals()["library"]()
        c = lbm_config()
        for name, _ in lbm_config._fields_:
            if name in ("cuda_stream", "dev_alloc", "dev_free", "alloc_ctx"):
                continue
            setattr(c, name, cfg.get(name, 0))
        self.cfg = dict(cfg)
        self._keep = []
        if stream is not None:
            c.cuda_stream = C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        if torch_allocator:
            import torch
            blocks = {}

            def _alloc(nbytes, stream_, ctx):
                t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
                blocks[t.data_ptr()] = t
                return t.data_ptr()

            def _free(ptr, stream_, ctx):
                blocks.pop(int(ptr), None)

            a, f = ALLOC_FN(_alloc), FREE_FN(_free)
            self._keep += [a, f, blocks]
            c.dev_alloc, c.dev_free = a, f
        h = C.c_void_p()
        create = self._lib.lbm_create_host if host_only else self._lib.lbm_create
        rc = create(C.byref(c), C.byref(h))
        if rc != 0:
            raise LBMError(rc, "lbm_create rejected the configuration")
        self._h = h
        self._cfg_struct = c

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise LBMError(rc, self._lib.lbm_last_error(self._h).decode())

    # -- API
    def set_geometry(self, loops):
        xy = np.ascontiguousarray(np.concatenate([np.asarray(p, dtype=np.float64) for p in loops])
                                  if loops else np.zeros((0, 2)))
        off = np.zeros(len(loops) + 1, dtype=np.int32)
        off[1:] = np.cumsum([len(p) for p in loops])
        self._check(self._lib.lbm_set_geometry(self._h, _dp(xy), _ip(off), len(loops)))
        self.n_loops = len(loops)

    def set_wall_slip(self, uw):
        uw = np.ascontiguousarray(uw, dtype=np.float64).reshape(-1)
        self._check(self._lib.lbm_set_wall_slip(self._h, _dp(uw), len(uw) // 2))

    def step(self, n=1):
        self._check(self._lib.lbm_step(self._h, int(n)))

    def step_async(self, n=1):
        self._check(self._lib.lbm_step_async(self._h, int(n)))

    def synchronize(self):
        self._check(self._lib.lbm_synchronize(self._h))

    def level_box(self, level):
        v = [C.c_int() for _ in range(4)]
        self._check(self._lib.lbm_get_level_box(self._h, level, *[C.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def mask(self, level):
        """Cell codes of a level over its box (also on host-only handles)."""
        i0, j0, nx, ny = self.level_box(level)
        mask = np.zeros((ny, nx), dtype=np.uint8)
        self._check(self._lib.lbm_get_fields(self._h, level, None, None, None, None,
                                             mask.ctypes.data_as(C.c_void_p), nx * ny))
        return mask

    def get_fields(self, level):
        i0, j0, nx, ny = self.level_box(level)
        rho, ux, uy, chi = (np.zeros((ny, nx)) for _ in range(4))
        mask = np.zeros((ny, nx), dtype=np.uint8)
        self._check(self._lib.lbm_get_fields(self._h, level, _dp(rho), _dp(ux), _dp(uy), _dp(chi),
                                             mask.ctypes.data_as(C.c_void_p), nx * ny))
        return dict(rho=rho, ux=ux, uy=uy, chi=chi, mask=mask, i0=i0, j0=j0)

    def get_populations(self, level):
        """Populations f_i of a level's box as an array (9, ny, nx); NaN where a cell has none."""
        i0, j0, nx, ny = self.level_box(level)
        pop = np.zeros((9, ny, nx))
        self._check(self._lib.lbm_get_populations(self._h, level, _dp(pop), pop.size))
        return pop

    def step_launch(self, level, kind):
        """lbm_step_launch: one launch of the level schedule (0 level step, 1 level step with
        restriction, 2 prolongation); the solver then refuses step() until set_state()."""
        self._check(self._lib.lbm_step_launch(self._h, int(level), int(kind)))

    def ghost_relay(self, level):
        """lbm_get_ghost_relay: band cells (n, 2) of a level and, per child m and direction i,
        the population its ghost child pulled in the fine level's last odd sub-step (n, 4, 9)."""
        n = C.c_int(0)
        self._check(self._lib.lbm_get_ghost_relay(self._h, level, None, None, 0, C.byref(n)))
        ij = np.zeros((max(n.value, 1), 2), dtype=np.int32)
        vals = np.zeros((max(n.value, 1), 4, 9))
        self._check(self._lib.lbm_get_ghost_relay(self._h, level, _ip(ij), _dp(vals), n.value, C.byref(n)))
        return ij[:n.value], vals[:n.value]

    def set_fields(self, level, rho=None, ux=None, uy=None, chi=None):
        i0, j0, nx, ny = self.level_box(level)
        arrs = [None if a is None else np.ascontiguousarray(np.broadcast_to(a, (ny, nx)), dtype=np.float64)
                for a in (rho, ux, uy, chi)]
        self._check(self._lib.lbm_set_fields(self._h, level, *[None if a is None else _dp(a) for a in arrs]))

    def get_loads(self):
        out = lbm_loads()
        n = C.c_int()
        self._check(self._lib.lbm_get_loads(self._h, C.byref(out), None, None, 0, C.byref(n)))
        cap = n.value
        cp, cf = np.zeros(max(cap, 1)), np.zeros(max(cap, 1))
        self._check(self._lib.lbm_get_loads(self._h, C.byref(out), _dp(cp), _dp(cf), cap, C.byref(n)))
        d = {k: getattr(out, k) for k, _ in lbm_loads._fields_}
        d["cp"], d["cf"] = cp[:cap], cf[:cap]
        return d

    def coefficients(self):
        """CL, CD, CDp, CDf, mass, dCL and step from one lbm_get_loads call (no per-segment arrays)."""
        out = lbm_loads()
        n = C.c_int()
        self._check(self._lib.lbm_get_loads(self._h, C.byref(out), None, None, 0, C.byref(n)))
        return {k: getattr(out, k) for k, _ in lbm_loads._fields_}

    def cut_links(self):
        n = C.c_int()
        self._check(self._lib.lbm_get_cut_links(self._h, None, None, 0, C.byref(n)))
        ijd = np.zeros((max(n.value, 1), 3), dtype=np.int32)
        q = np.zeros(max(n.value, 1))
        self._check(self._lib.lbm_get_cut_links(self._h, _ip(ijd), _dp(q), n.value, C.byref(n)))
        return ijd[:n.value], q[:n.value]

    def wall_records(self):
        n = C.c_int()
        self._check(self._lib.lbm_get_wall_records(self._h, None, None, None, 0, C.byref(n)))
        m = max(n.value, 1)
        ij, geo, ns = np.zeros((m, 2), dtype=np.int32), np.zeros((m, 9)), np.zeros(m, dtype=np.int32)
        self._check(self._lib.lbm_get_wall_records(self._h, _ip(ij), _dp(geo), _ip(ns), n.value, C.byref(n)))
        return ij[:n.value], geo[:n.value], ns[:n.value]

    def wall_stencils(self):
        """(sij [n, 16, 2], wr [n, 16], wu [n, 16]): reference-point stencils and weights."""
        n = C.c_int()
        self._check(self._lib.lbm_get_wall_stencils(self._h, None, None, None, 0, C.byref(n)))
        sij = np.zeros((n.value, 16, 2), dtype=np.int32)
        wr, wu = np.zeros((n.value, 16)), np.zeros((n.value, 16))
        self._check(self._lib.lbm_get_wall_stencils(self._h, _ip(sij), _dp(wr), _dp(wu), n.value, C.byref(n)))
        return sij, wr, wu

    def segment_map(self):
        """(mid [n, 2], b12 [n, 2], w12 [n, 2]): wall segments -> two nearest wall records."""
        n = C.c_int()
        self._check(self._lib.lbm_get_segment_map(self._h, None, None, None, 0, C.byref(n)))
        mid, w12 = np.zeros((n.value, 2)), np.zeros((n.value, 2))
        b12 = np.zeros((n.value, 2), dtype=np.int32)
        self._check(self._lib.lbm_get_segment_map(self._h, _dp(mid), _ip(b12), _dp(w12), n.value, C.byref(n)))
        return mid, b12, w12

    def wall_state(self):
        n = C.c_int()
        self._check(self._lib.lbm_get_wall_state(self._h, None, 0, C.byref(n)))
        st = np.zeros((max(n.value, 1), 8))
        self._check(self._lib.lbm_get_wall_state(self._h, _dp(st), n.value, C.byref(n)))
        return st[:n.value]

    def prolong_independence(self):
        """lbm_get_prolong_independence: per level, whether its prolongation may share a launch
        with that of the level above."""
        out = (C.c_int * 16)()
        self._check(self._lib.lbm_get_prolong_independence(self._h, out, 16))
        return [bool(out[l]) for l in range(self.cfg["levels"])]

    def work_list(self, level, warps=False):
        """lbm_get_work_list: (n, 3) int array of the level kernel's work tiles or warps in
        launch order: global i, j of the tile's first cell, warp (-1 for tiles)."""
        n = C.c_int()
        w = int(bool(warps))
        self._check(self._lib.lbm_get_work_list(self._h, level, w, None, 0, C.byref(n)))
        out = np.zeros((max(n.value, 1), 3), dtype=np.int32)
        self._check(self._lib.lbm_get_work_list(self._h, level, w, out.ctypes.data_as(C.c_void_p), n.value, C.byref(n)))
        return out[:n.value]

    def flags(self, level):
        """The level kernel's 32-bit flag word per cell of the level box."""
        i0, j0, nx, ny = self.level_box(level)
        f = np.zeros((ny, nx), dtype=np.uint32)
        self._check(self._lib.lbm_get_flags(self._h, level, f.ctypes.data_as(C.POINTER(C.c_uint)), nx * ny))
        return f

    def wall_distance(self, level):
        i0, j0, nx, ny = self.level_box(level)
        d = np.zeros((ny, nx))
        self._check(self._lib.lbm_get_wall_distance(self._h, level, _dp(d), nx * ny))
        return d

    def info(self):
        out = lbm_info()
        self._check(self._lib.lbm_get_info(self._h, C.byref(out)))
        L = out.levels
        return dict(levels=L, cells_active=list(out.cells_active[:L]), cells_present=list(out.cells_present[:L]),
                    slots=list(out.slots[:L]), node_updates_per_step=out.node_updates_per_step,
                    wall_records=out.wall_records, cut_links=out.cut_links,
                    surface_segments=out.surface_segments, kernels_per_step=out.kernels_per_step,
                    bytes_per_node_update=out.bytes_per_node_update, device_bytes=out.device_bytes,
                    work_tiles=list(out.work_tiles[:L]), work_warps=list(out.work_warps[:L]))

    def autotune(self, steps=10):
        """lbm_autotune: per-level register budget and PDL choice by timing; advances the
        solve by the returned steps_taken coarse steps."""
        out = lbm_tune_report()
        self._check(self._lib.lbm_autotune(self._h, int(steps), C.byref(out)))
        return _tune_dict(out)

    def get_state(self) -> np.ndarray:
        """lbm_get_state: the solve's state at the current step as a uint8 array."""
        n = C.c_size_t()
        self._check(self._lib.lbm_get_state(self._h, None, 0, C.byref(n)))
        buf = np.empty(n.value, dtype=np.uint8)
        self._check(self._lib.lbm_get_state(self._h, buf.ctypes.data_as(C.c_void_p), buf.size, C.byref(n)))
        return buf

    def set_state(self, blob):
        """lbm_set_state: continue from a blob of get_state (same configuration and grid)."""
        b = np.ascontiguousarray(blob, dtype=np.uint8)
        self._check(self._lib.lbm_set_state(self._h, b.ctypes.data_as(C.c_void_p), b.size))

    def set_launch_variant(self, min_blocks, pdl=1, sched=None, shape=None):
        """lbm_set_launch_variant: per-level register budget (5 or 6 blocks per SM), grid
        schedule (SCHED_TILE, SCHED_PERSIST, SCHED_WARPS or SCHED_WARPS4), work shape of a warp
        (0 a 16 x 2 block, 1 a 32-cell row; 0 with the warp-list schedules) and PDL."""
        mb = np.ascontiguousarray(min_blocks, dtype=np.int32)
        pe = np.ascontiguousarray(sched if sched is not None else [SCHED_TILE] * len(mb), dtype=np.int32)
        sh = np.ascontiguousarray(shape if shape is not None else [0] * len(mb), dtype=np.int32)
        self._check(self._lib.lbm_set_launch_variant(self._h, _ip(mb), _ip(pe), _ip(sh), int(pdl)))

    def set_load_history(self, every, capacity=1024):
        """lbm_set_load_history: eq 30's coefficients and the mass into a device ring every
        `every` coarse steps (0 stops)."""
        self._check(self._lib.lbm_set_load_history(self._h, int(every), int(capacity)))

    def load_history(self):
        """lbm_get_load_history: the kept records, oldest first, as dicts."""
        n = C.c_int()
        self._check(self._lib.lbm_get_load_history(self._h, None, 0, C.byref(n)))
        arr = (lbm_load_record * max(n.value, 1))()
        self._check(self._lib.lbm_get_load_history(self._h, C.cast(arr, C.c_void_p), n.value, C.byref(n)))
        return [{k: getattr(arr[i], k) for k, _ in lbm_load_record._fields_} for i in range(n.value)]

    def set_timeline(self, on=True):
        """lbm_set_timeline: per-block clock records in every launch of the step graphs."""
        self._check(self._lib.lbm_set_timeline(self._h, int(bool(on))))

    def timeline(self):
        """lbm_get_timeline: per launch of the last run of each step graph: graph, level, kind
        (0 even, 1 odd, 2 prolongation), blocks, t_wait_us, t_end_us."""
        n = C.c_int()
        self._check(self._lib.lbm_get_timeline(self._h, None, 0, C.byref(n)))
        arr = (lbm_launch_time * max(n.value, 1))()
        self._check(self._lib.lbm_get_timeline(self._h, C.cast(arr, C.c_void_p), n.value, C.byref(n)))
        return [{k: getattr(arr[i], k) for k, _ in lbm_launch_time._fields_} for i in range(n.value)]

    def set_prolong_merge(self, on=True):
        """lbm_set_prolong_merge: one launch for the prolongations of consecutive levels where
        they are independent; returns the number of levels whose prolongation can join."""
        n = C.c_int()
        self._check(self._lib.lbm_set_prolong_merge(self._h, int(bool(on)), C.byref(n)))
        return n.value

    def time_kernels(self, n=1):
        out = lbm_kernel_times()
        self._check(self._lib.lbm_time_kernels(self._h, int(n), C.byref(out)))
        return {out.name[i].value.decode(): dict(ms=out.total_ms[i], launches=out.launches[i], cells=out.cells[i])
                for i in range(out.n_classes)}


def _tune_dict(out):
    L = out.levels
    cand = list(zip(out.candidate_min_blocks, out.candidate_sched, out.candidate_shape))
    return dict(levels=L, candidates=cand,
                level_us={c: list(out.level_us[i][:L]) for i, c in enumerate(cand)},
                min_blocks=list(out.min_blocks[:L]), sched=list(out.sched[:L]),
                shape=list(out.shape[:L]),
                step_us_confirm={"pick": out.step_us_confirm[0], "pick_tile_for_persistent": out.step_us_confirm[1],
                                 "before": out.step_us_confirm[2],
                                 **{("uniform",) + c: out.step_us_confirm[3 + i] for i, c in enumerate(cand)}},
                confirm_choice=out.confirm_choice,
                default_step_us=out.default_step_us,
                step_us={"pdl_off": out.step_us[0], "pdl_on": out.step_us[1]}, pdl=out.pdl,
                steps_taken=out.steps_taken)


def level_mass_noalloc(flags, drho, ux, uy, chi, n_cells, area, mass_out, nonfinite_out, stream=0):
    """lbm_level_mass_noalloc on caller-owned device buffers given as raw device addresses
    (for example ``tensor.data_ptr()``); returns the status code.  Only enqueues work."""
    return library().lbm_level_mass_noalloc(flags, drho, ux, uy, chi, int(n_cells), float(area), mass_out,
                                            nonfinite_out, stream)


class Batch:
    """lbm_batch: steps several resident solves in lockstep, one launch per level-schedule
    node covering every member (see include/lbm.h).  The solvers stay owned by the caller
    and must outlive the batch; queries go to the solvers themselves."""

    def __init__(self, solvers):
        self._lib = library()
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[s._h for s in self.solvers])
        h = C.c_void_p()
        rc = self._lib.lbm_batch_create(arr, len(self.solvers), C.byref(h))
        if rc != 0:
            raise LBMError(rc, "lbm_batch_create")
        self._h = h

    def step(self, n=1):
        rc = self._lib.lbm_batch_step(self._h, int(n))
        if rc != 0:
            raise LBMError(rc, "lbm_batch_step: " + self._lib.lbm_batch_last_error(self._h).decode())

    def info(self):
        m, lv, nk = C.c_int(), C.c_int(), C.c_longlong()
        self._lib.lbm_batch_info(self._h, C.byref(m), C.byref(lv), C.byref(nk))
        return dict(members=m.value, levels=lv.value, kernels_per_step=nk.value)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
