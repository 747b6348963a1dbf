"""The bounds-checked debug build (libklb_checked.so, -DKLB_CHECK_BOUNDS).

Every kernel of that build compares each global index it forms (state
buffers, dense field arrays, diagnostics rings, the adjoint's buffers) with
the extent of its buffer; an index out of range is skipped and flagged, and
klb_sync reports KLB_E_BOUNDS.  Nothing traps, so a fault of the index
arithmetic shows up as an error code with the context intact.

* The probe entry point plants one guarded store past the end of a buffer:
  the checked build reports it, the ordinary build refuses the call.
* The edge-size parity tests (grids narrower than a tile, one tile, ragged
  tiles, every boundary kind, both FP32 tile shapes, FP64), the batch test
  and the adjoint's dot-product tests run unchanged on the checked build, in a
  child process: no index falls outside its buffer and the results still
  match the oracle.
"""
import os
import subprocess
import sys

import pytest

from paper_1010_4124_gb300 import inputs, klb

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _checked_env():
    env = dict(os.environ)
    env["KLB_CHECKED"] = "1"
    return env


def test_probe_refused_by_the_ordinary_build():
    pb = inputs.khi(40, 24, 1)
    with klb.Klb.from_problem(pb, precision="fp32") as h:
        assert klb.lib().klb_debug_bounds_probe(h.h) == -1


def test_probe_is_flagged_by_the_checked_build():
    code = r"""
from paper_1010_4124_gb300 import inputs, klb
pb = inputs.khi(40, 24, 1)
with klb.Klb.from_problem(pb, precision="fp32") as h:
    h.init_fields(*inputs.fields(pb))
    assert klb.lib().klb_debug_bounds_probe(h.h) == 0
    assert klb.lib().klb_sync(h.h) == -8, "the out-of-range store was not flagged"
    assert klb.lib().klb_sync(h.h) == 0, "the flag was not cleared"
    h.step(2)
    h.sync()
print("probe flagged")
"""
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=_checked_env(), capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0 and "probe flagged" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]


def test_edge_parity_tests_pass_on_the_checked_build():
    tests = ["tests/test_gpu_step.py::test_fp32_one_step_parity_every_size",
             "tests/test_gpu_step.py::test_fp64_one_step_parity",
             "tests/test_gpu_step.py::test_fp32_variants_are_bitwise_identical",
             "tests/test_gpu_step.py::test_diagnostics_series_parity",
             "tests/test_gpu_batch.py",
             "tests/test_gpu_adjoint.py::test_dot_product_with_oracle_tangent"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", *tests], cwd=ROOT,
                       env=_checked_env(), capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
