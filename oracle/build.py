"""Compile the CPU oracle (oracle.c) into oracle/_build/liboracle.so.

Test infrastructure only: called by the tests, the smoke check and the
benchmark's CPU-baseline leg, and by the package build step so that the
checker exists on a fresh machine.  Plain gcc; OpenMP when available.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")

# -ffp-contract=off: no fused multiply-add, so the rounding of every
# operation is the one written in oracle.c (gcc contracts by default on
# aarch64 otherwise).  No -ffast-math: sums keep their written order.
BASE_FLAGS = ["-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-std=c11"]


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc"] + BASE_FLAGS + ["-fopenmp", SRC, "-o", tmp, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        # no OpenMP runtime: the single-threaded build gives identical results
        cmd = ["gcc"] + BASE_FLAGS + [SRC, "-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
