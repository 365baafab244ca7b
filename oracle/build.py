"""Compiles the CPU oracle (oracle.c) into liboracle_f32.so and liboracle_f64.so.

Test infrastructure: the oracle is loaded only by the tests, the smoke check and the
benchmark's CPU-baseline leg.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
FLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-Wall", "-Wno-unused-function"]


def lib_path(real):
    return os.path.join(HERE, f"liboracle_{real}.so")


def build(force=False, extra=()):
    src = os.path.join(HERE, "oracle.c")
    deps = [src] + [os.path.join(HERE, f) for f in ("oracle_project.inc", "oracle_partition.inc", "oracle_levels.inc", "oracle_ssim.inc")]
    for real, ctype in (("f32", "float"), ("f64", "double")):
        out = lib_path(real)
        if (not force and os.path.exists(out)
                and os.path.getmtime(out) >= max(os.path.getmtime(d) for d in deps)):
            continue
        cmd = ["gcc", *FLAGS, *extra, f"-DREAL={ctype}", "-o", out + ".tmp", src, "-lm"]
        subprocess.check_call(cmd)
        os.replace(out + ".tmp", out)


if __name__ == "__main__":
    build(force="--force" in sys.argv)
