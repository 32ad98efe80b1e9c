"""Build libgsc.so in place with nvcc for sm_103a (B300)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libgsc.so")
BUILD_DIR = os.path.join(HERE, "_build")
# The bounds-checked variant (GSC_DEBUG_BOUNDS): data-indexed stores test
# their index against the buffer's capacity, flag ERR_BOUNDS and skip; a
# substitute for a device memory checker, selected by a process through the
# GSC_LIBRARY environment variable.
LIB_CHECKED = os.path.join(HERE, "libgsc_checked.so")

SOURCES = ["api.cu", "frame_cull.cu", "derive_f32.cu", "derive_unfused.cu", "derive_tc.cu", "project.cu", "cache.cu", "sort.cu", "raster.cu", "reuse.cu", "noalloc_scan.cu", "probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-Xcompiler", "-ffp-contract=off", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    deps += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False, checked: bool = False) -> str:
    """libgsc.so, or with checked=True the bounds-checked libgsc_checked.so."""
    bdir = os.path.join(BUILD_DIR, "checked") if checked else BUILD_DIR
    out = LIB_CHECKED if checked else LIB
    defs = ["-DGSC_DEBUG_BOUNDS"] if checked else []
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    objs = []
    changed = force or not os.path.exists(out)
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(bdir, s + ".o")
        objs.append(obj)
        if force or _stale(obj, src):
            cmd = [nvcc, *ARCH, *FLAGS, *defs, "-c", src, "-o", obj]
            if ptxas_v:
                cmd.insert(1, "-Xptxas=-v")
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            subprocess.check_call(cmd)
            changed = True
    if changed:
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", out + ".tmp", *objs]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        os.replace(out + ".tmp", out)
    return out


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_v="-v" in sys.argv, checked="--checked" in sys.argv)
