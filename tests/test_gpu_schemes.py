"""Parity of the lower-order convection schemes (first-order upwind,
second-order upwind, second-order TVD; Sec. III.B, Fig. 2) between the CUDA
step, through the C ABI, and the FP64 oracle: FP64 <= 1e-12 per plane, FP32
<= 1e-5 on rho, u, T of smooth data; both FP32 tile shapes and the batched
engine give identical bits."""
import numpy as np
import pytest

from gpu_common import gpu_handle, oracle_params, perturbed_state, rel_err_fields, rel_err_planes
from oracle import core
from paper_1010_4124_gb300 import inputs, klb

pytestmark = pytest.mark.gpu

LOW = ("upwind1", "upwind2", "tvd")


def _problem(nx, ny, bcx, bcy, dt=2e-5, tau=4e-5, dx=0.01, dy=0.012):
    return inputs.Problem("custom", nx, ny, dx, dy, dt, tau, 1, bc_x=(bcx, bcx), bc_y=(bcy, bcy))


@pytest.mark.parametrize("scheme", LOW)
@pytest.mark.parametrize("bcx,bcy", [("periodic", "outflow"), ("fixed_eq", "periodic"), ("outflow", "fixed_eq")])
def test_fp64_parity_rough_data(scheme, bcx, bcy):
    pb = _problem(67, 45, bcx, bcy)
    p = oracle_params(pb, scheme=scheme)
    fields = inputs.rough_random_fields(67, 45, seed=5)
    f0 = perturbed_state(pb, fields, seed=6)
    ref, _ = core.run(p, f0, 20, fixed=core.fixed_ghosts(p, *fields))
    with gpu_handle(pb, "fp64", scheme=scheme) as h:
        h.init_fields(*[np.ascontiguousarray(a) for a in fields])
        h.set_f(np.ascontiguousarray(f0))
        h.step(20)
        got = h.get_f()
    assert rel_err_planes(got, ref) <= 1e-12


@pytest.mark.parametrize("scheme", ("upwind1", "tvd"))
def test_fp64_sod_full_run(scheme):
    # the Sod tube of the Fig. 2 comparison (200 x 4, 5000 steps to t = 0.1)
    pb = inputs.sod(200, 4, 5000)
    p = oracle_params(pb, scheme=scheme)
    fields = inputs.fields(pb)
    ref, _ = core.run(p, core.init_feq(p, *fields), pb.steps, fixed=core.fixed_ghosts(p, *fields))
    with gpu_handle(pb, "fp64", scheme=scheme) as h:
        h.init_fields(*fields)
        h.step(pb.steps)
        got = h.get_f()
    errs = rel_err_fields(got, ref, p)
    assert max(errs.values()) <= 1e-12, errs


@pytest.mark.parametrize("scheme", LOW)
def test_fp32_smooth_data(scheme):
    pb = inputs.Problem("smooth", 128, 96, 0.002, 0.002, 1e-5, 1e-5, 300)
    p = oracle_params(pb, scheme=scheme)
    fields = inputs.smooth_random_fields(128, 96, seed=8, amp=0.08)
    ref, _ = core.run(p, core.init_feq(p, *fields), pb.steps)
    got = []
    for v in (0, 1):
        with gpu_handle(pb, "fp32", scheme=scheme) as h:
            h.variant = v
            h.init_fields(*fields)
            h.step(pb.steps)
            got.append(h.get_f())
    assert np.array_equal(got[0], got[1])
    errs = rel_err_fields(got[0], ref, p)
    assert errs["rho"] <= 1e-5 and errs["u"] <= 1e-5 and errs["T"] <= 1e-5, errs


def test_batch_with_a_lower_order_scheme_equals_single_grids():
    pbs = [inputs.khi(nx, ny, 30, sample_every=10) for nx, ny in ((96, 64), (64, 80), (128, 48))]
    fl = [inputs.fields(pb) for pb in pbs]
    with klb.KlbBatch.from_problems(pbs, scheme="tvd") as bt:
        for m, f in zip(bt.members, fl):
            m.init_fields(*f)
        bt.step(30)
        bt.sync()
        got = [m.get_f() for m in bt.members]
    for pb, f, g in zip(pbs, fl, got):
        with gpu_handle(pb, "fp32", scheme="tvd") as h:
            h.variant = 1
            h.init_fields(*f)
            h.step(30)
            assert np.array_equal(h.get_f(), g)
