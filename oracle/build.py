"""Compile the FP64 CPU oracle (test infrastructure only).

Produces oracle/liboklb.so (real = double) and oracle/liboklb_cs.so
(real = double _Complex, for complex-step tangents) from oracle/oklb.c with
gcc, OpenMP over rows and no floating-point contraction, so that the oracle
rounds every operation exactly as written.
"""
import fcntl
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oklb.c")
FLAGS = ["-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11"]


def _fresh(out: str) -> bool:
    return os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC)


def build(force: bool = False) -> None:
    outs = (("liboklb.so", []), ("liboklb_cs.so", ["-DOKLB_COMPLEX"]))
    if not force and all(_fresh(os.path.join(HERE, n)) for n, _ in outs):
        return
    # processes that start together build one at a time; each library is
    # written under a temporary name and renamed into place
    with open(os.path.join(HERE, ".build.lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        for name, extra in outs:
            out = os.path.join(HERE, name)
            if not force and _fresh(out):
                continue
            tmp = out + ".tmp"
            subprocess.run(["gcc", *FLAGS, *extra, "-o", tmp, SRC, "-lm"], check=True)
            os.replace(tmp, out)


if __name__ == "__main__":
    build(force="--force" in sys.argv)
