"""Builds libcgs.so (the CUDA library behind include/cgs.h) in-tree for sm_103a.

Each .cu file is compiled to an object with nvcc; the files whose floating-point results
decide integers (the projection key path, LoD selection, MAD bounds) are compiled with
-fmad=false so that no multiply-add is contracted; the compositing backward is built with
flush-to-zero.  The objects are linked into one shared library next to this file.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcgs.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
          "-I", CSRC, "--expt-relaxed-constexpr"]
NO_FMA = {"project.cu", "project_bwd.cu", "select.cu", "partition.cu", "levels.cu"}
FTZ = {"render_bwd.cu"}  # gradient arithmetic only; the decisions it shares with the forward are pinned in PTX
SOURCES = ["api.cu", "select.cu", "project.cu", "sort.cu", "render.cu", "render_bwd.cu", "project_bwd.cu",
           "static_ws.cu", "partition.cu", "levels.cu", "ssim.cu", "peaks.cu", "boundary.cu"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def build(force=False, verbose=False, extra=()):
    os.makedirs(BUILD, exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "cgs.h")]
    newest = max(os.path.getmtime(d) for d in deps)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    objs = []
    nvcc = _nvcc()
    for src in SOURCES:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        flags = list(COMMON) + list(extra)
        if src in NO_FMA:
            flags.append("-fmad=false")
        if src in FTZ:
            flags.append("-ftz=true")
        cmd = [nvcc, *ARCH, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        objs.append(obj)
    tmp = LIB + ".tmp"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [])
