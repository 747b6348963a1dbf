"""The C-ABI library builds, loads and exports every entry point declared in
include/klb.h (no compute calls: this runs without a GPU)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(klb_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1010_4124_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_exports_every_declared_symbol(lib):
    names = _declared("klb.h")
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_params_default_is_host_only(lib):
    from paper_1010_4124_gb300 import klb
    p = klb.klb_params()
    klb.lib().klb_params_default(C.byref(p))
    assert tuple(p.v) == (1.0, 2.0, 3.0)
    assert p.eps == 1e-6 and p.precision == 0 and p.stream is None


def test_params_struct_layout_matches_header(lib):
    # the ctypes mirror must have the same size as the C struct: compile a
    # probe with the host compiler against include/klb.h
    import subprocess
    import tempfile
    from paper_1010_4124_gb300 import klb
    src = '#include "klb.h"\n#include <stdio.h>\n#include <stddef.h>\nint main(void){printf("%zu %zu %zu\\n", sizeof(klb_params), offsetof(klb_params, stream), offsetof(klb_params, scheme));return 0;}\n'
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "p")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        size, off, off_s = map(int, subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split())
    assert C.sizeof(klb.klb_params) == size
    assert klb.klb_params.stream.offset == off
    assert klb.klb_params.scheme.offset == off_s


def test_create_rejects_bad_params_without_gpu(lib):
    from paper_1010_4124_gb300 import klb
    p = klb.make_params(0, 8, 0.01, 0.01, 1e-5, 1e-5)
    with pytest.raises(klb.KlbError) as e:
        klb.Klb(p)
    assert e.value.code == -1
    p = klb.make_params(8, 8, 0.01, 0.01, 1e-5, 1e-5, bc_x=("periodic", "outflow"))
    with pytest.raises(klb.KlbError) as e:
        klb.Klb(p)
    assert e.value.code == -1
    p = klb.make_params(8, 8, 0.01, 0.01, 1e-5, 1e-5, v=(1.0, 1.0, 3.0))
    with pytest.raises(klb.KlbError) as e:
        klb.Klb(p)
    assert e.value.code == -1
    # an empty grid and non-positive step sizes
    for args in ((8, 0, 0.01, 0.01, 1e-5, 1e-5), (8, 8, 0.01, 0.01, 0.0, 1e-5), (8, 8, 0.01, 0.01, 1e-5, -1.0),
                 (8, 8, 0.0, 0.01, 1e-5, 1e-5)):
        with pytest.raises(klb.KlbError) as e:
            klb.Klb(klb.make_params(*args))
        assert e.value.code == -1, args


def test_scheme_validation_without_gpu(lib):
    # an unknown convection scheme is refused before any device work; a batch
    # must share one scheme; the adjoint differentiates the WENO5 step only
    from paper_1010_4124_gb300 import klb
    p = klb.make_params(8, 8, 0.01, 0.01, 1e-5, 1e-5)
    p.scheme = 7
    with pytest.raises(klb.KlbError) as e:
        klb.Klb(p)
    assert e.value.code == -1 and "scheme" in str(e.value)
    ps = [klb.make_params(8, 8, 0.01, 0.01, 1e-5, 1e-5, scheme=s) for s in ("tvd", "upwind1")]
    with pytest.raises(klb.KlbError) as e:
        klb.KlbBatch(ps)
    assert e.value.code == -1
    q = klb.make_params(8, 8, 0.01, 0.01, 1e-5, 1e-5, scheme="upwind1", sample_every=1)
    with pytest.raises(klb.KlbError) as e:
        klb.KlbAdjoint(q, 4, 2)
    assert e.value.code == -1


def test_binding_refuses_arrays_of_the_wrong_size():
    # the library reads or writes exactly n elements through each pointer; the
    # binding checks the count before any call (a shorter array would be read
    # past its end)
    from paper_1010_4124_gb300 import klb
    a = np.zeros((4, 5))
    assert klb._ptr(a, 20) == (a.ctypes.data, 0)
    with pytest.raises(ValueError):
        klb._ptr(a, 21)
    with pytest.raises(ValueError):
        klb._ptr(np.zeros(19 * 20 - 1), 19 * 20)
    with pytest.raises(TypeError):
        klb._ptr(np.zeros(20, dtype=np.float32), 20)
    with pytest.raises(TypeError):
        klb._ptr(np.zeros((5, 4)).T, 20)  # not C-contiguous
    torch = pytest.importorskip("torch")
    t = torch.zeros(20, dtype=torch.float64)
    assert klb._ptr(t, 20) == (t.data_ptr(), 0)
    with pytest.raises(ValueError):
        klb._ptr(t, 19)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # the product path has no fallback: without the CUDA library every call
    # raises (nothing is computed on the CPU)
    from paper_1010_4124_gb300 import klb
    monkeypatch.setattr(klb, "_lib", None)
    monkeypatch.setattr(klb, "LIB_PATH", str(tmp_path / "libklb.so"))
    with pytest.raises(RuntimeError, match="not built"):
        klb.lib()
    with pytest.raises(RuntimeError):
        klb.Klb(klb.make_params(8, 8, 0.01, 0.01, 1e-5, 1e-5))


def test_fp32_weno_eps_below_the_range_is_refused(lib):
    # klb_create validates before touching the device: an FP32 WENO5 handle
    # whose 3/4 eps / max(v)^2 is below 2e-19 (squared smoothness indicators
    # below the normal FP32 range) is refused with KLB_E_INVAL
    from paper_1010_4124_gb300 import klb
    p = klb.make_params(32, 32, 0.002, 0.002, 1e-5, 1e-5, precision="fp32", eps=1e-18)
    h = C.c_void_p()
    assert klb.lib().klb_create(C.byref(p), C.byref(h)) == -1
    assert b"eps" in klb.lib().klb_last_error(None)
