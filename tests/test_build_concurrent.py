"""Builds started together (the ranks of one job each call the build) run one
at a time and leave a usable library: three processes force-rebuild the
oracle at once."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_concurrent_oracle_builds_leave_a_loadable_library():
    code = "import sys; sys.path.insert(0, %r); from oracle import build; build.build(force=True)" % ROOT
    procs = [subprocess.Popen([sys.executable, "-c", code], cwd=ROOT) for _ in range(3)]
    assert all(p.wait(timeout=300) == 0 for p in procs)
    check = ("import sys; sys.path.insert(0, %r); from oracle import core; import numpy as np; "
             "print(core.Fk(1.0)[1])" % ROOT)
    r = subprocess.run([sys.executable, "-c", check], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and abs(float(r.stdout) - 1 / 9) < 1e-12, r.stderr
