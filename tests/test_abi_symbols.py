"""The product library loads on any host and exports every entry point that
include/lbm.h declares (no compute calls: those need a GPU)."""
import ctypes
import os
import re

import paper_2601_18443_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for required in ("lbm_create", "lbm_set_geometry", "lbm_step", "lbm_get_fields", "lbm_get_loads",
                     "lbm_destroy", "lbm_set_fields", "lbm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    pkg.build()
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2601_18443_gb300", "_build", "liblbm.so"))
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    from paper_2601_18443_gb300 import _build_ext
    monkeypatch.setattr(_build_ext, "SO", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pkg, "_lib", None)
    try:
        pkg.library()
    except RuntimeError as e:
        assert "not built" in str(e)
    else:  # pragma: no cover
        raise AssertionError("library() must raise when liblbm.so is missing")


def test_create_rejects_invalid_configurations():
    # validation happens on the host before any CUDA call
    from paper_2601_18443_gb300 import workloads as W
    bad = [dict(levels=0), dict(levels=17), dict(nx0=2), dict(h0=0.0), dict(layers=2), dict(Re=0.0),
           dict(Ma=-1.0), dict(chord=0.0), dict(store=7), dict(periodic=1, nx0=48), dict(wall_model=5),
           dict(outlet=2), dict(outlet=-1)]
    for kw in bad:
        cfg = W.base_config(**kw)
        try:
            pkg.Solver(cfg)
        except pkg.LBMError as e:
            assert e.code == -1, (kw, e.code)
        else:  # pragma: no cover
            raise AssertionError(f"accepted invalid configuration {kw}")
