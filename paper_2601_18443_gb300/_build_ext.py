"""Builds the in-tree CUDA library liblbm.so for sm_103a (nvcc + g++, no cmake)."""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
SO = os.path.join(OUT_DIR, "liblbm.so")
SO_CHECK = os.path.join(OUT_DIR, "liblbm_check.so")   # LBM_BOUNDS_CHECK build
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm.so")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)) + [os.path.join(INCLUDE, "lbm.h")]


def up_to_date(so: str = SO) -> bool:
    if not os.path.exists(so):
        return False
    t = os.path.getmtime(so)
    return all(os.path.getmtime(f) <= t for f in _sources())


def build(force: bool = False, verbose: bool = False, bounds_check: bool = False) -> str:
    """Build liblbm.so, or with bounds_check liblbm_check.so: the same library with every
    table-derived index of the level step checked on the device (LBM_BOUNDS_CHECK)."""
    so = SO_CHECK if bounds_check else SO
    if not force and up_to_date(so):
        return so
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    tag = f".{os.getpid()}" + (".check" if bounds_check else "")
    objs = {name: os.path.join(OUT_DIR, name.rsplit(".", 1)[0] + tag + ".o")
            for name in ("grid.cpp", "kernels.cu", "lbm_capi.cu", "noalloc.cu")}
    cuflags = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fopenmp",
               "-Xptxas", "-v" if verbose else "-O3"] + ARCH + (["-DLBM_BOUNDS_CHECK"] if bounds_check else [])
    cmds = [
        ["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", "-ffp-contract=off", "-c",
         os.path.join(CSRC, "grid.cpp"), "-o", objs["grid.cpp"]],
        [nvcc] + cuflags + ["-c", os.path.join(CSRC, "kernels.cu"), "-o", objs["kernels.cu"]],
        [nvcc] + cuflags + ["-c", os.path.join(CSRC, "lbm_capi.cu"), "-o", objs["lbm_capi.cu"]],
        [nvcc] + cuflags + ["-c", os.path.join(CSRC, "noalloc.cu"), "-o", objs["noalloc.cu"]],
    ]
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for c in cmds]
    logs = []
    for c, p in zip(cmds, procs):
        out, _ = p.communicate()
        logs.append(out)
        if p.returncode != 0:
            raise RuntimeError("compile failed: " + " ".join(c) + "\n" + out)
    if verbose:
        print("\n".join(logs))
    tmp = so + tag
    link = [nvcc, "-shared"] + ARCH + ["-o", tmp] + list(objs.values()) + ["-Xcompiler", "-fopenmp", "-lgomp"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: " + " ".join(link) + "\n" + r.stdout)
    os.replace(tmp, so)
    for o in objs.values():
        os.remove(o)
    return so
