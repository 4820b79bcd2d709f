"""Build libfv3.so (the C-ABI of include/fv3.h) for sm_103a with nvcc.

Translation units are compiled in parallel into ``_build/`` next to this file
and linked into ``_build/libfv3.so``; nothing is installed elsewhere.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libfv3.so")
# (source, object name, defines): fv3_kernels.cu is three units, one per
# precision plus the shared host code, so the heavy kernels build in parallel
SOURCES = [("fv3_grid.cpp", "fv3_grid", ()),
           ("fv3_kernels.cu", "fv3_kernels_f64", ("-DFV3_TU=64",)),
           ("fv3_kernels.cu", "fv3_kernels_f32", ("-DFV3_TU=32",)),
           ("fv3_kernels.cu", "fv3_kernels_f32m64", ("-DFV3_TU=33",)),
           ("fv3_kernels.cu", "fv3_kernels_main", ("-DFV3_TU=1",)),
           ("fv3_capi.cu", "fv3_capi", ()), ("fv3_calib.cu", "fv3_calib", ()),
           ("fv3_noalloc.cu", "fv3_noalloc", ()), ("fv3_mlp.cu", "fv3_mlp", ()),
           ("fv3_remap.cu", "fv3_remap", ()), ("fv3_exchange.cu", "fv3_exchange", ())]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "fv3.h"))
    return files


def _compile(unit, extra):
    src, name, defs = unit
    obj = os.path.join(OUT, name + ".o")
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
           "-I", os.path.join(ROOT, "include"), "-I", CSRC, *defs, *extra, "-c",
           os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd.insert(1, "-x")
        cmd.insert(2, "cu")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (name, " ".join(cmd), r.stderr))
    return obj, r.stderr


def build(force=False, verbose=False, extra=()):
    os.makedirs(OUT, exist_ok=True)
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(f) <= t for f in _deps()):
            return LIB
    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        res = list(ex.map(lambda s: _compile(s, list(extra)), SOURCES))
    if verbose:
        for _, err in res:
            if err:
                print(err)
    objs = [o for o, _ in res]
    tmp = LIB + ".tmp"
    r = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="-f" in sys.argv, verbose=True,
                extra=("-Xptxas", "-v") if "-v" in sys.argv else ()))
