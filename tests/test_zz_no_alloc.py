"""The allocation-free diagnostics entry point, klb_diagnostics_static.

It serves callers that cannot allocate device memory while they run (an
application whose memory manager owns every device allocation, a service whose
device footprint is fixed after start-up, a latency-bound loop that cannot
afford cudaMalloc's synchronisation): its partial sums live in a fixed device
array of the library
instead of a cudaMalloc'ed buffer.  Its results must equal those of the
handle-based path (klb_diagnostics), on two calls in a row.  This file is
collected last so that a failure here does not hide any other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1010_4124_gb300 import inputs, klb

PREC = {"fp32": 0, "fp64": 1}


def _call(f_ptr, prec, nx, ny, pitch, plane, v, out_ptr, stream=None):
    vv = (C.c_double * 3)(*v)
    return klb.lib().klb_diagnostics_static(f_ptr, PREC[prec], nx, ny, pitch, plane, C.cast(vv, C.c_void_p),
                                            out_ptr, stream)


@pytest.mark.gpu
@pytest.mark.parametrize("prec,variant", [("fp32", None), ("fp32", 0), ("fp64", None)])
def test_static_diagnostics_equal_the_handle_path(prec, variant):
    # variant None: the handle keeps the tile shape it starts with (32 x 8
    # tiles for this size), whose reduction runs in another order than the
    # static path's 32 x 16 tiles: equal to rounding.  variant 0: the handle's
    # reduction uses the same tiles and order as the static path: equal bit
    # for bit.
    torch = pytest.importorskip("torch")
    pb = inputs.khi(300, 170, 0, Dv=3.0, Drho=5.0, sample_every=1)
    out = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda")
    with klb.Klb.from_problem(pb, precision=prec) as h:
        if variant is not None:
            h.variant = variant
        h.init_fields(*inputs.fields(pb))
        for _ in range(2):  # two calls in a row, on two successive states
            h.step(5)
            ref = h.diagnostics()[-1]  # the existing entry point: sample of the current state (synchronises)
            base, pitch, plane, gx, gy = h.layout()
            assert (gx, gy) == (4, 3)
            code = _call(base, prec, pb.nx, pb.ny, pitch, plane, pb.v, out.data_ptr())
            assert code == 0, klb.lib().klb_diagnostics_static_error()
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            if variant == 0:
                assert np.array_equal(got, ref), (got, ref)
            for k in range(7):
                # momentum sums cancel to ~0: measure them on the mass scale
                scale = abs(ref[0]) if k in (1, 2) else abs(ref[k])
                assert abs(got[k] - ref[k]) <= 1e-12 * scale, (k, got[k], ref[k])
            out.fill_(float("nan"))


def test_static_diagnostics_reject_sizes_beyond_the_scratch():
    # an FP64 state of 2048 x 2048 needs 64 x 256 = 16384 partial records; the
    # fixed scratch holds 4096: rejected before any device work
    nx = ny = 2048
    pitch = (nx + 7 + 31) // 32 * 32
    plane = pitch * (ny + 6)
    code = _call(C.c_void_p(16), "fp64", nx, ny, pitch, plane, (1.0, 2.0, 3.0), C.c_void_p(16))
    assert code == -1
    assert b"4096" in klb.lib().klb_diagnostics_static_error()
    code = _call(None, "fp64", 8, 8, 64, 64 * 14, (1.0, 2.0, 3.0), C.c_void_p(16))
    assert code == -1
    # a row pitch beyond the int range of the kernels' row arithmetic
    code = _call(C.c_void_p(16), "fp32", 8, 8, 1 << 31, (1 << 31) * 14, (1.0, 2.0, 3.0), C.c_void_p(16))
    assert code == -1 and b"pitch" in klb.lib().klb_diagnostics_static_error()
    # an FP32 grid of 2^24 tiles of 32 x 16 nodes (1024 tile columns x 16384
    # tile rows): beyond the exact range of the tile index split
    nx, ny = 32768 - 4, 16 * 16384
    pitch = (nx + 7 + 31) // 32 * 32
    code = _call(C.c_void_p(16), "fp32", nx, ny, pitch, pitch * (ny + 6), (1.0, 2.0, 3.0), C.c_void_p(16))
    assert code == -1 and b"2^24" in klb.lib().klb_diagnostics_static_error()
