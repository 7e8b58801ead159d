"""Build libnlem.so (sm_103a) in-tree with nvcc: one object per translation unit, compiled in
parallel, then linked into paper_1501_03879_gb300/lib/libnlem.so.  build(debug=True) builds the
same sources with -DNLEM_DEBUG (the bounds checks of csrc/debug.h; relocatable device code, so that
every translation unit records into one device record) into lib/libnlem_debug.so."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OBJ = os.path.join(ROOT, "_build", "obj")
OBJ_DEBUG = os.path.join(ROOT, "_build", "obj_debug")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libnlem.so")
LIB_DEBUG = os.path.join(LIBDIR, "libnlem_debug.so")
DEBUG_FLAGS = ["-DNLEM_DEBUG", "-rdc=true"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return hs + [os.path.join(ROOT, "include", "nlem.h")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, debug: bool = False) -> str:
    objdir, lib = (OBJ_DEBUG, LIB_DEBUG) if debug else (OBJ, LIB)
    extra = DEBUG_FLAGS if debug else []
    os.makedirs(objdir, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    hdrs = headers()
    jobs = []
    objs = []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + hdrs):
            cmd = ["nvcc", *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    failed = []
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or ptxas_info or r.returncode:
                sys.stdout.write(r.stdout)
                sys.stdout.write(r.stderr)
            if r.returncode:
                failed.append(cmd[-3])
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(failed))
    if force or jobs or _stale(lib, objs):
        cmd = ["nvcc", *ARCH, *(["-rdc=true"] if debug else []), "-shared", "-o", lib, *objs, "-lcudart"]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv, debug="--debug" in sys.argv)
