"""The one JSON line of bench.py, for both arms: the keys and types the
benchmark contract names.  The reference arm (the FP64 oracle on the host
cores) runs on the CPU; our arm needs the GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COMMON = {"metric": str, "value": (int, float), "unit": str, "n_gpus": int, "steps": int, "warmup": int,
          "ms_per_step": (int, float), "higher_is_better": bool, "scaling": str, "dtype": str, "data": str,
          "config": dict, "cpu_baseline": dict, "e2e": dict}


def _line(args):
    r = subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def _check_common(d):
    for k, t in COMMON.items():
        assert k in d and isinstance(d[k], t), k
    assert d["value"] > 0 and d["higher_is_better"] is True and d["scaling"] == "weak"
    assert "workload" in d["config"]
    assert d["vs_baseline"] is None  # the paper publishes no timing
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in d["e2e"], k
    for k in ("value", "unit", "cores", "kind", "sample"):
        assert k in d["cpu_baseline"], k
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1


def test_reference_arm_line():
    d = _line(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    _check_common(d)
    assert d["impl"] == "reference" and d["dtype"] == "f64"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


@pytest.mark.gpu
def test_our_arm_line():
    d = _line(["--workload", "khi512", "--steps", "20", "--warmup", "3", "--no-sweep", "--no-adjoint",
               "--no-schemes", "--no-physics"])
    _check_common(d)
    assert d["dtype"] == "f32" and d["gpu_launches"] >= 1
    for key in ("roofline", "roofline_hbm"):
        r = d[key]
        for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
            assert k in r, (key, k)
        assert 0 < r["frac"] < 1.5 and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3
    assert d["roofline"]["bound"] == "alu" and d["roofline_hbm"]["bound"] == "hbm"
    c = d["clocks"]
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(c)
