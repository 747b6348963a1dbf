"""Parity of the CUDA step (through the C ABI) with the FP64 CPU oracle.

Tolerances (max norm, relative to each field's or plane's max norm):
FP64 <= 1e-12 per field after any number of steps; FP32 (arithmetic in FP32,
diagnostics in FP64) <= 1e-5 on rho, u, T after 1000 steps of smooth data.
"""
import os
import tempfile

import numpy as np
import pytest

from gpu_common import gpu_handle, oracle_params, perturbed_state, rel_err_fields, rel_err_global, rel_err_planes
from oracle import core
from paper_1010_4124_gb300 import inputs, klb

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


def _problem(nx, ny, bcx, bcy, dt=2e-5, tau=4e-5, dx=0.01, dy=0.012):
    return inputs.Problem("custom", nx, ny, dx, dy, dt, tau, 1, bc_x=(bcx, bcx), bc_y=(bcy, bcy))


BCS = [("periodic", "periodic"), ("periodic", "outflow"), ("outflow", "periodic"), ("fixed_eq", "outflow"),
       ("outflow", "fixed_eq"), ("fixed_eq", "fixed_eq")]
SIZES = [(70, 37), (32, 8), (5, 3), (1, 1), (97, 130)]


@pytest.mark.parametrize("bcx,bcy", BCS)
@pytest.mark.parametrize("nx,ny", SIZES)
def test_fp64_one_step_parity(nx, ny, bcx, bcy):
    pb = _problem(nx, ny, bcx, bcy)
    p = oracle_params(pb)
    fields = inputs.rough_random_fields(nx, ny, seed=nx * 1000 + ny)
    f0 = perturbed_state(pb, fields, seed=3)
    fixed = core.fixed_ghosts(p, *fields)
    ref = core.step(p, f0, fixed=fixed)
    with gpu_handle(pb, "fp64") as h:
        h.init_fields(*[np.ascontiguousarray(a) for a in fields])
        h.set_f(np.ascontiguousarray(f0))
        h.step(1)
        got = h.get_f()
    assert rel_err_planes(got, ref) <= TOL64


@pytest.mark.parametrize("bcx,bcy", BCS[:4])
def test_fp64_many_steps_parity(bcx, bcy):
    pb = _problem(67, 45, bcx, bcy)
    p = oracle_params(pb)
    fields = inputs.smooth_random_fields(67, 45, seed=8, amp=0.08)
    f0 = perturbed_state(pb, fields, seed=4, amp=0.02)
    fixed = core.fixed_ghosts(p, *fields)
    ref, _ = core.run(p, f0, 60, fixed=fixed)
    with gpu_handle(pb, "fp64") as h:
        h.init_fields(*[np.ascontiguousarray(a) for a in fields])
        h.set_f(np.ascontiguousarray(f0))
        h.step(60)
        got = h.get_f()
    errs = rel_err_fields(got, ref, p)
    assert max(errs.values()) <= TOL64, errs


def test_sod_fp64_full_run():
    # config: Sod tube 200 x 4, dt = tau = 2e-5, 5000 steps to t = 0.1
    pb = inputs.sod(200, 4, 5000)
    p = oracle_params(pb)
    fields = inputs.fields(pb)
    f0 = core.init_feq(p, *fields)
    ref, _ = core.run(p, f0, pb.steps, fixed=core.fixed_ghosts(p, *fields))
    with gpu_handle(pb, "fp64") as h:
        h.init_fields(*fields)
        h.step(pb.steps)
        got = h.get_f()
        assert h.step_count == 5000
    errs = rel_err_fields(got, ref, p)
    assert max(errs.values()) <= TOL64, errs


def test_fp32_smooth_1000_steps():
    # smooth periodic data (a few low Fourier modes around (1, 0.1, -0.05, 1)),
    # dx = dy = 0.002, dt = tau = 1e-5: FP32 within 1e-5 of the FP64 oracle
    # on rho, u and T after 1000 steps
    pb = inputs.Problem("smooth", 128, 96, 0.002, 0.002, 1e-5, 1e-5, 1000)
    p = oracle_params(pb)
    fields = inputs.smooth_random_fields(128, 96, seed=8, amp=0.08)
    f0 = core.init_feq(p, *fields)
    ref, _ = core.run(p, f0, 1000)
    with gpu_handle(pb, "fp32") as h:
        h.init_fields(*fields)
        h.step(1000)
        got = h.get_f()
    errs = rel_err_fields(got, ref, p)
    assert errs["rho"] <= TOL32 and errs["u"] <= TOL32 and errs["T"] <= TOL32, errs


def test_fp32_khi_fields_1000_steps():
    # the KHI shear layer (tanh over 4 cells, WENO weights far from optimal):
    # FP32 fields after 1000 steps, bound recorded at 1e-4 (measured ~3e-5)
    pb = inputs.khi(128, 128, 1000, Dv=4.0, Drho=4.0)
    p = oracle_params(pb)
    fields = inputs.fields(pb)
    ref, _ = core.run(p, core.init_feq(p, *fields), 1000)
    with gpu_handle(pb, "fp32") as h:
        h.init_fields(*fields)
        h.step(1000)
        got = h.get_f()
    errs = rel_err_fields(got, ref, p)
    print("fp32 khi 128^2 after 1000 steps:", errs)
    assert max(errs["rho"], errs["u"], errs["T"]) <= 1e-4, errs


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_diagnostics_series_parity(prec, tol):
    # tol is the field bar (relative to the field's max norm); the sums of
    # mass, momentum and energy (columns 0-3) are held to it.  Columns 4-6 are
    # built from u_y alone (max |u_y|, max and sum of rho u_y^2 / 2): an error
    # of tol max|u| in u_y is tol max|u| / max|u_y| of max |u_y| and twice that
    # of rho u_y^2 / 2 -- about 2.5e-4 and 5e-4 here in FP32 (max|u| = 0.25,
    # max |u_y| >= 0.0099 over the series)
    pb = inputs.khi(64, 96, 200, Dv=4.0, Drho=4.0, sample_every=10)
    p = oracle_params(pb)
    fields = inputs.fields(pb)
    f0 = core.init_feq(p, *fields)
    _, dref = core.run(p, f0, pb.steps, sample_every=10)
    with gpu_handle(pb, prec) as h:
        h.init_fields(*fields)
        h.step(pb.steps)
        d = h.diagnostics()
    assert d.shape == dref.shape == (21, 7)
    umax = np.abs(fields[1]).max()
    uy_over_u = dref[:, 4].min() / umax  # the smallest max|u_y| of the series against max|u|
    for k in range(7):
        scale = np.abs(dref[:, k]).max()
        if k in (1, 2):  # momentum sums cancel to ~0: compare against the mass scale
            scale = np.abs(dref[:, 0]).max()
        bound = tol if k <= 3 else (tol / uy_over_u if k == 4 else 2 * tol / uy_over_u)
        assert np.abs(d[:, k] - dref[:, k]).max() <= bound * scale, (k, bound)


@pytest.mark.parametrize("variant", [0, 1])
def test_fp32_diagnostics_equal_the_oracle_sums_of_the_same_state(variant):
    # The FP32 diagnostics (FP32 node values, compensated FP32 partial sums,
    # FP64 across warps and CTAs) against the oracle's FP64 diagnostics of the
    # very same FP32 state (read back exactly): every interior node counted
    # once on ragged tiles (one node missed would be 1.7e-6 of the mass), the
    # sums accurate to the rounding of the node values.  Sample 0 is reduced
    # inside the first step's kernel, sample 1 by the stand-alone kernel.
    pb = inputs.khi(1000, 600, 10, Dv=4.0, Drho=4.0, sample_every=10)
    p = oracle_params(pb)
    with gpu_handle(pb, "fp32") as h:
        h.variant = variant
        h.init_fields(*inputs.fields(pb))
        f0 = h.get_f()
        h.step(10)
        f1 = h.get_f()
        d = h.diagnostics()
    assert d.shape == (2, 7)
    for got, f in ((d[0], f0), (d[1], f1)):
        ref = core.diag(p, f)
        mass = abs(ref[0])
        assert abs(got[0] - ref[0]) <= 1e-8 * mass, (got[0], ref[0])
        assert abs(got[1] - ref[1]) <= 1e-6 * mass and abs(got[2] - ref[2]) <= 1e-6 * mass
        assert abs(got[3] - ref[3]) <= 1e-6 * abs(ref[3])
        for k in (4, 5, 6):
            assert abs(got[k] - ref[k]) <= 1e-5 * abs(ref[k]), (k, got[k], ref[k])


def test_conservation_fp64_periodic():
    pb = _problem(80, 72, "periodic", "periodic")
    fields = inputs.smooth_random_fields(80, 72, seed=2, amp=0.1)
    f0 = perturbed_state(pb, fields, seed=9, amp=0.02)
    with gpu_handle(pb, "fp64", sample_every=50) as h:
        h.init_fields(*fields)
        h.set_f(np.ascontiguousarray(f0))
        h.step(200)
        d = h.diagnostics()
    # samples after 0, 50, ..., 200 steps; the first is taken after set_f
    for k, scale in ((0, d[0, 0]), (1, d[0, 0]), (2, d[0, 0]), (3, d[0, 3])):
        assert np.abs(d[:, k] - d[0, k]).max() <= 200 * 1e-14 * abs(scale), k


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_khi512_full_size_step_parity(prec, tol):
    # the 512 x 512 KHI at full size: after 200 GPU steps, one oracle step from
    # the GPU state must equal the GPU's next step at every node
    pb = inputs.khi(512, 512, 200)
    p = oracle_params(pb)
    with gpu_handle(pb, prec) as h:
        h.init_fields(*inputs.fields(pb))
        h.step(200)
        fa = h.get_f()
        h.step(1)
        fb = h.get_f()
    ref = core.step(p, fa)
    if prec == "fp64":
        assert rel_err_planes(fb, ref) <= tol
    else:
        assert rel_err_global(fb, ref) <= tol
        errs = rel_err_fields(fb, ref, p)
        assert max(errs["rho"], errs["u"], errs["T"]) <= tol, errs


def test_roofline_4096_windows_parity():
    # the 4096 x 4096 four-mode KHI in FP32: windows of the GPU state after 20
    # steps; one oracle step on each window (periodic wrap, then the 3-node rim
    # discarded) equals the GPU's next step on the window's core
    pb = inputs.roofline_4096(20)
    rng = np.random.default_rng(12)
    with gpu_handle(pb, "fp32") as h:
        h.init_fields(*inputs.fields(pb))
        h.step(20)
        fa = h.get_f()
        h.step(1)
        fb = h.get_f()
    W = 40
    corners = [(0, 0), (4096 - W, 4096 - W), (2048 - W // 2, 2048 - W // 2)] + \
        [tuple(rng.integers(0, 4096 - W, 2)) for _ in range(3)]
    for (y0, x0) in corners:
        ys = np.arange(y0 - 3, y0 + W + 3)
        xs = np.arange(x0 - 3, x0 + W + 3) % 4096
        win = fa[:, :, xs]
        # rows: inside the domain use the state, beyond it the outflow copy
        win = win[:, np.clip(ys, 0, 4095), :]
        pw = core.Params(nx=W + 6, ny=W + 6, dx=pb.dx, dy=pb.dy, dt=pb.dt, tau=pb.tau,
                         bc_x=("periodic", "periodic"), bc_y=("periodic", "periodic"))
        ref = core.step(pw, win)[:, 3:-3, 3:-3]
        got = fb[:, y0:y0 + W, x0:x0 + W]
        assert rel_err_global(got, ref) <= 1e-5, (y0, x0)
        pc = core.Params(nx=W, ny=W, dx=pb.dx, dy=pb.dy, dt=pb.dt, tau=pb.tau)
        errs = rel_err_fields(got, ref, pc)
        assert max(errs["rho"], errs["u"], errs["T"]) <= 1e-5, ((y0, x0), errs)


class _DeviceState:
    """The current FP32 state of a handle as a device array [19][rows][pitch]
    (rows = ghost rows included), for torch to view without a copy."""

    def __init__(self, h):
        base, pitch, plane, self.gx, self.gy = h.layout()
        self.__cuda_array_interface__ = {"shape": (19, plane // pitch, pitch), "typestr": "<f4",
                                         "data": (base, False), "version": 3, "strides": None}


def test_fp32_step_beyond_2g_elements_windows_parity():
    # 16384 x 16384 FP32: 5.1 G elements per buffer (offsets past 2^31), 41 GB
    # of state.  The KHI fields are built on the device; windows of the state
    # (with a 3-node rim) are read through the library's layout before and
    # after one more step, and one oracle step on each window equals the GPU's
    # step on the window's core (rows beyond the domain: the outflow copy).
    torch = pytest.importorskip("torch")
    n, W = 16384, 40
    pb = inputs.khi(n, n, 3, Dv=16.0, Drho=16.0)
    dev = torch.device("cuda")
    y = ((torch.arange(n, device=dev, dtype=torch.float64) - n / 2 + 0.5) * pb.dy)[:, None]
    x = (torch.arange(n, device=dev, dtype=torch.float64) * pb.dx)[None, :]
    th = torch.tanh(y / (16.0 * pb.dy))
    rho = (3.0 + 2.0 * th).expand(n, n).contiguous()
    ux = (0.25 * th).expand(n, n).contiguous()
    T = (1.5 / rho).contiguous()
    uy = (0.01 * torch.sin(2 * np.pi * x / (n * pb.dx)) * torch.exp(-(y / (0.05 * n * pb.dy)) ** 2)).contiguous()
    del th
    rng = np.random.default_rng(16384)
    corners = [(0, 0), (n - W, n - W), (n // 2 - W // 2, n // 2 - W // 2), (0, n - W)] + \
        [tuple(int(v) for v in rng.integers(0, n - W, 2)) for _ in range(3)]

    def windows(h, rim):
        st = torch.as_tensor(_DeviceState(h), device=dev)
        out = []
        for (y0, x0) in corners:
            ys = torch.as_tensor(np.clip(np.arange(y0 - rim, y0 + W + rim), 0, n - 1) + 3, device=dev)
            xs = torch.as_tensor(np.arange(x0 - rim, x0 + W + rim) % n + 4, device=dev)
            out.append(st.index_select(1, ys).index_select(2, xs).double().cpu().numpy())
        return out

    with gpu_handle(pb, "fp32") as h:
        h.init_fields(rho, ux, uy, T)
        h.sync()  # the fields are read on the handle's stream
        del rho, ux, uy, T
        h.step(2)
        h.sync()
        _, _, _, gx, gy = h.layout()
        assert (gx, gy) == (4, 3)
        fa = windows(h, 3)
        h.step(1)
        h.sync()
        fb = windows(h, 0)
    for (y0, x0), wa, got in zip(corners, fa, fb):
        pw = core.Params(nx=W + 6, ny=W + 6, dx=pb.dx, dy=pb.dy, dt=pb.dt, tau=pb.tau,
                         bc_x=("periodic", "periodic"), bc_y=("periodic", "periodic"))
        ref = core.step(pw, wa)[:, 3:-3, 3:-3]
        assert rel_err_global(got, ref) <= 1e-5, (y0, x0)
        errs = rel_err_fields(got, ref, core.Params(nx=W, ny=W, dx=pb.dx, dy=pb.dy, dt=pb.dt, tau=pb.tau))
        assert max(errs["rho"], errs["u"], errs["T"]) <= 1e-5, ((y0, x0), errs)


def test_step_before_init_and_bad_args():
    pb = _problem(16, 16, "periodic", "periodic")
    with gpu_handle(pb, "fp32") as h:
        with pytest.raises(klb.KlbError) as e:
            h.step(1)
        assert e.value.code == -6
        h.init_fields(*inputs.smooth_random_fields(16, 16, 0))
        with pytest.raises(klb.KlbError) as e:
            h.step(-1)
        assert e.value.code == -1


def test_zero_steps_and_empty_series():
    # zero steps enqueue nothing and leave the state, the step count and the
    # (unsampled) diagnostics series as they are; an empty batch is refused
    pb = _problem(16, 12, "periodic", "outflow")
    for prec in ("fp32", "fp64"):
        with gpu_handle(pb, prec, sample_every=0) as h:
            h.init_fields(*inputs.smooth_random_fields(16, 12, 1))
            f0, n0 = h.get_f(), h.launch_count
            h.step(0)
            h.sync()
            assert h.launch_count == n0 and h.step_count == 0
            assert np.array_equal(h.get_f(), f0)
            assert h.diagnostics().shape == (0, 7)
    with klb.KlbBatch.from_problems([pb]) as b:
        b.members[0].init_fields(*inputs.smooth_random_fields(16, 12, 1))
        b.step(0)
        b.sync()
        assert b.members[0].step_count == 0
    with pytest.raises((klb.KlbError, ValueError)):
        klb.KlbBatch([])


def test_diagnostics_ring_keeps_the_latest_samples():
    # a ring of 5 samples after 11 samples (every 2 of 20 steps) holds the last
    # 5, bitwise those of a large ring, and returns them oldest first (the copy
    # runs across the ring's wrap); asking for 3 gives the oldest 3 of them
    pb = _problem(20, 14, "periodic", "outflow")
    fields = inputs.smooth_random_fields(20, 14, 4)
    series = {}
    for cap in (5, 64):
        with gpu_handle(pb, "fp32", sample_every=2, diag_capacity=cap) as h:
            h.init_fields(*fields)
            h.step(20)
            series[cap] = (h.diagnostics(), h.diagnostics(cap=3))
    assert series[64][0].shape == (11, 7) and series[5][0].shape == (5, 7)
    assert np.array_equal(series[5][0], series[64][0][-5:])
    assert np.array_equal(series[5][1], series[64][0][-5:-2])


def test_bounded_wait_runs_out_and_context_survives():
    # fault injection from the host: the step kernel also waits on a barrier
    # nothing arrives on, with a short poll budget; the wait runs out, the
    # kernel reports KLB_E_DEVICE_TIMEOUT and exits cleanly
    pb = _problem(64, 48, "periodic", "outflow")
    fields = inputs.smooth_random_fields(64, 48, 1)
    with gpu_handle(pb, "fp32") as h:
        h.init_fields(*fields)
        h.debug_inject_wait_timeout(64)
        h.step(3)
        with pytest.raises(klb.KlbError) as e:
            h.sync()
        assert e.value.code == -5
        # the context is still usable: a fresh handle steps normally
    with gpu_handle(pb, "fp64") as h2:
        h2.init_fields(*fields)
        h2.step(2)
        h2.sync()
        p = oracle_params(pb)
        ref, _ = core.run(p, core.init_feq(p, *fields), 2)
        assert rel_err_planes(h2.get_f(), ref) <= TOL64


def test_nonfinite_state_is_reported():
    pb = _problem(40, 40, "periodic", "periodic")
    fields = [np.array(a) for a in inputs.smooth_random_fields(40, 40, 1)]
    fields[0][7, 11] = np.nan  # a NaN planted in the initial density
    pb.sample_every = 1
    with gpu_handle(pb, "fp32") as h:
        h.init_fields(*fields)
        h.step(2)
        with pytest.raises(klb.KlbError) as e:
            h.diagnostics()
        assert e.value.code == -4


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_save_load_resumes_bitwise(prec):
    pb = inputs.khi(96, 80, 40, sample_every=10)
    fields = inputs.fields(pb)
    with gpu_handle(pb, prec) as a:
        a.init_fields(*fields)
        a.step(40)
        fa, da = a.get_f(), a.diagnostics()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.klb")
        with gpu_handle(pb, prec) as b:
            b.init_fields(*fields)
            b.step(20)
            b.save(path)
        with gpu_handle(pb, prec) as c:
            c.load(path)
            assert c.step_count == 20
            c.step(20)
            fc, dc = c.get_f(), c.diagnostics()
    assert np.array_equal(fa, fc)
    assert np.array_equal(da, dc)


def test_device_pointer_fields_from_torch():
    torch = pytest.importorskip("torch")
    pb = inputs.khi(64, 64, 10)
    fields = inputs.fields(pb)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in fields]
    with gpu_handle(pb, "fp64") as h:
        h.init_fields(*dev)
        h.step(10)
        out = tuple(torch.empty((64, 64), dtype=torch.float64, device="cuda") for _ in range(4))
        h.moments(out)
        host = h.moments()
    for a, b in zip(out, host):
        assert np.array_equal(a.cpu().numpy(), b)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_khi512_growth_rate_matches_oracle(prec):
    # the single 512 x 512 KHI run, 4000 steps sampled every 10: the growth
    # rate fitted from the GPU's diagnostics is within 1% of the oracle's
    # (stored by tests/golden/make_khi_gamma.py, which calls only oracle/)
    import json
    from oracle import fit
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "khi512_gamma.json")))
    pb = inputs.khi(512, 512, 4000, Dv=4.0, Drho=4.0, sample_every=10)
    with gpu_handle(pb, prec) as h:
        h.init_fields(*inputs.fields(pb))
        h.step(pb.steps)
        d = h.diagnostics()
    dref = np.array(gold["diag"])
    assert d.shape == dref.shape
    g = fit.growth_rates(d, pb.dt, pb.sample_every)
    for got, key in zip(g, ("gamma_ln_max_uy", "gamma_half_ln_max_Ex", "gamma_half_ln_sum_Ex")):
        assert abs(got - gold[key]) <= 0.01 * abs(gold[key]), (key, got, gold[key])
    if prec == "fp64":
        for k in range(7):
            scale = np.abs(dref[:, 0 if k in (1, 2) else k]).max()
            assert np.abs(d[:, k] - dref[:, k]).max() <= 1e-12 * scale, k


def test_fp32_default_tile_shape_by_size():
    # a new FP32 handle starts with the shape measured faster for its size:
    # 8-row tiles while the grid has at most 40 sixteen-row tiles per SM
    torch = pytest.importorskip("torch")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for nx, ny in ((256, 256), (1024, 512), (2048, 1024), (2048, 2048), (4096, 4096)):
        tiles16 = ((nx + 4 + 31) // 32) * ((ny + 15) // 16)
        with gpu_handle(inputs.khi(nx, ny, 1), "fp32") as h:
            assert h.variant == (1 if tiles16 <= 40 * sms else 0), (nx, ny, h.variant)
    with gpu_handle(inputs.khi(64, 64, 1), "fp64") as h:
        assert h.variant == 0


@pytest.mark.parametrize("bcx,bcy", [("periodic", "outflow"), ("outflow", "fixed_eq")])
def test_fp32_variants_are_bitwise_identical(bcx, bcy):
    # the two tile shapes of the FP32 kernel compute every node with the same
    # arithmetic: the states agree bit for bit (ghost images and fixed ghosts
    # included)
    pb = inputs.khi(300, 170, 30).with_(bc_x=(bcx, bcx), bc_y=(bcy, bcy))
    fields = inputs.fields(pb)
    out = []
    for v in (0, 1):
        with gpu_handle(pb, "fp32") as h:
            h.variant = v
            assert h.variant == v
            h.init_fields(*fields)
            h.step(30)
            out.append(h.get_f())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_mean_density_profile(prec, tol):
    # the averaged density profile (Sec. IV.A) of the state the CUDA path
    # reaches: equal to the oracle's profile of that same state (summation
    # order only), and to the profile of the oracle's own run
    pb = inputs.khi(96, 64, 50, Dv=3.0, Drho=5.0)
    p = oracle_params(pb)
    fields = inputs.fields(pb)
    ref, _ = core.run(p, core.init_feq(p, *fields), 50)
    with gpu_handle(pb, prec) as h:
        h.init_fields(*fields)
        h.step(50)
        md = h.mean_density()
        got = h.get_f()
        import torch
        dev = torch.empty(pb.ny, dtype=torch.float64, device="cuda")
        h.mean_density(dev)
        np.testing.assert_array_equal(dev.cpu().numpy(), md)
    np.testing.assert_allclose(md, core.mean_density(p, got), rtol=1e-13)
    np.testing.assert_allclose(md, core.mean_density(p, ref), rtol=tol)


@pytest.mark.parametrize("bcx,bcy", BCS)
@pytest.mark.parametrize("nx,ny", SIZES + [(28, 16), (29, 17), (60, 33)])
def test_fp32_one_step_parity_every_size(nx, ny, bcx, bcy):
    # one FP32 step from rough data, both tile shapes, against the FP64 oracle
    # on the scale of f: grids narrower than one tile, exactly one tile (28 + 4
    # ghost columns = 32), ragged last tiles in x and y, every boundary kind
    pb = _problem(nx, ny, bcx, bcy)
    p = oracle_params(pb)
    fields = inputs.rough_random_fields(nx, ny, seed=nx * 7 + ny)
    f0 = perturbed_state(pb, fields, seed=5)
    ref = core.step(p, f0, fixed=core.fixed_ghosts(p, *fields))
    got = []
    for v in (0, 1):
        with gpu_handle(pb, "fp32") as h:
            h.variant = v
            h.init_fields(*[np.ascontiguousarray(a) for a in fields])
            h.set_f(np.ascontiguousarray(f0))
            h.step(1)
            got.append(h.get_f())
    assert np.array_equal(got[0], got[1])
    assert rel_err_global(got[0], ref) <= 2e-6


@pytest.mark.parametrize("sample_every", [0, 10, 7])
def test_graph_replayed_steps_equal_single_launches(sample_every):
    # klb_step replays runs of steps from a CUDA graph (FP32 WENO5, runs of at
    # least 64 steps starting at a sampling point); stepping one call per step
    # never does.  Both must give the same states and diagnostics, bit for bit,
    # including runs that start off a sampling point and a ragged remainder.
    pb = inputs.khi(96, 80, 0, sample_every=sample_every)
    fields = inputs.fields(pb)
    out = []
    for graphs in (True, False):
        with gpu_handle(pb, "fp32", sample_every=sample_every) as h:
            h.init_fields(*fields)
            if graphs:
                h.step(3)
                h.step(200)
                h.step(157)
            else:
                for _ in range(360):
                    h.step(1)
            assert h.step_count == 360
            out.append((h.get_f(), h.diagnostics() if sample_every else None))
    assert np.array_equal(out[0][0], out[1][0])
    if sample_every:
        assert np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_pinned_host_fields_and_moments_equal_pageable(prec):
    # pinned host arrays are read (init) and written (moments) by the kernels
    # directly across the host link; pageable ones go through device staging:
    # the same states and moments either way
    torch = pytest.importorskip("torch")
    pb = inputs.khi(90, 70, 15)
    fields = [np.ascontiguousarray(a) for a in inputs.fields(pb)]
    pinned = [torch.from_numpy(a.copy()).pin_memory() for a in fields]
    out = []
    for src in ("pageable", "pinned"):
        with gpu_handle(pb, prec) as h:
            h.init_fields(*(fields if src == "pageable" else [p.numpy() for p in pinned]))
            h.step(pb.steps)
            f = h.get_f()
            if src == "pageable":
                m = h.moments()
            else:
                m = tuple(torch.empty((pb.ny, pb.nx), dtype=torch.float64).pin_memory() for _ in range(4))
                h.moments(tuple(t.numpy() for t in m))
                m = tuple(t.numpy() for t in m)
            out.append((f, [np.array(a) for a in m]))
    assert np.array_equal(out[0][0], out[1][0])
    for a, b in zip(out[0][1], out[1][1]):
        assert np.array_equal(a, b)
