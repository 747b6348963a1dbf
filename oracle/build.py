"""Compile the FP64 CPU oracle (test infrastructure only).

Produces oracle/liboklb.so (real = double) and oracle/liboklb_cs.so
(real = double _Complex, for complex-step tangents) from oracle/oklb.c with
gcc, OpenMP over rows and no floating-point contraction, so that the oracle
rounds every operation exactly as written.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oklb.c")
FLAGS = ["-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11"]


def build(force: bool = False) -> None:
    for name, extra in (("liboklb.so", []), ("liboklb_cs.so", ["-DOKLB_COMPLEX"])):
        out = os.path.join(HERE, name)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
            continue
        cmd = ["gcc", *FLAGS, *extra, "-o", out, SRC, "-lm"]
        subprocess.run(cmd, check=True)


if __name__ == "__main__":
    build(force="--force" in sys.argv)
