"""Host-side logic: the workload recipes and their differentiable torch copy."""
import numpy as np
import pytest

from paper_1010_4124_gb300 import inputs


def test_torch_khi_recipe_matches_numpy():
    torch = pytest.importorskip("torch")
    from paper_1010_4124_gb300.adjoint import khi_fields_torch
    pb = inputs.khi(40, 30, 10, Dv=3.0, Drho=5.0)
    uy0 = inputs.perturbation_shape(pb)
    a = inputs.fields(pb)
    b = khi_fields_torch(pb, 3.0, 5.0, uy0)
    for x, y in zip(a, b):
        np.testing.assert_allclose(y.numpy(), x, rtol=1e-15, atol=1e-16)


def test_sweep_instances_are_seeded_and_complete():
    a = inputs.sweep_instances(10)
    b = inputs.sweep_instances(10)
    assert len(a) == 32
    assert [(p.nx, p.ny) for p in a] == [(p.nx, p.ny) for p in b]
    assert {(p.Dv, p.Drho) for p in a} == {(float(v), float(r)) for v in inputs.SWEEP_DV for r in inputs.SWEEP_DRHO}
    assert {(p.nx, p.ny) for p in a} <= set(inputs.SWEEP_SIZES)


def test_sod_recipe():
    pb = inputs.sod(200, 4, 5000)
    rho, ux, uy, T = inputs.fields(pb)
    assert rho[0, 99] == 1.0 and rho[0, 100] == 0.125
    assert T[0, 99] == 1.0 and T[0, 100] == 0.8
    assert pb.dt == 2e-5 and pb.tau == 2e-5 and pb.steps * pb.dt == pytest.approx(0.1)


def test_roofline_workload_phases_are_seeded():
    pb = inputs.roofline_4096(1)
    np.testing.assert_array_equal(inputs.phases(pb), inputs.phases(inputs.roofline_4096(5)))
    assert pb.nx == pb.ny == 4096 and pb.Dv == pb.Drho == 16.0 and pb.modes == 4
