"""Build libaxp.so (the CUDA library behind include/axp.h) for sm_103a with nvcc.

Each translation unit is compiled in parallel and linked into
paper_2406_16796_gb300/_lib/libaxp.so.  The general-path unit is compiled
without multiply-add contraction (its FP64 results follow a literal
double-precision evaluation of the scheme); the others use the default.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libaxp.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# host code is compiled without multiply-add contraction as well (gcc contracts by
# default on some hosts), so host-side FP64 set-up values do not depend on the host
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
          "-I", INCLUDE, "-I", CSRC]
# per-unit extra flags
UNITS = {
    "api.cu": [],
    "kernels_general.cu": ["--fmad=false"],
    "kernels_diag.cu": [],
    "kernels_init.cu": [],
    "kernels_fused.cu": [],
    "kernels_fused_f64.cu": [],
    "kernels_fused_f32.cu": [],
    "batch1d.cu": [],
    "group2d.cu": [],
    "particles.cu": [],
}


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libaxp")


def _sources():
    return [os.path.join(CSRC, u) for u in UNITS]


def _deps():
    deps = _sources()
    for d in (CSRC, INCLUDE):
        deps += [os.path.join(d, f) for f in os.listdir(d) if f.endswith((".h", ".cuh"))]
    return deps


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    obj_dir = os.path.join(OUT_DIR, "obj")
    os.makedirs(obj_dir, exist_ok=True)
    cc = nvcc()

    def compile_one(unit):
        src = os.path.join(CSRC, unit)
        obj = os.path.join(obj_dir, unit.replace(".cu", ".o"))
        cmd = [cc] + ARCH + COMMON + UNITS[unit] + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (unit, " ".join(cmd), r.stderr))
        if verbose and r.stderr.strip():
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + ".tmp"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose=True))
