"""Pins of the oracle's diagnostics and growth-rate fit (Sec. IV of the paper)."""
import numpy as np
import pytest

from oracle import core, fit
from paper_1010_4124_gb300 import inputs


def test_diag_matches_fields_by_brute_force():
    p = core.Params(nx=9, ny=7, dx=0.01, dy=0.01, dt=1e-5, tau=1e-5)
    fl = inputs.rough_random_fields(p.nx, p.ny, 3)
    f = core.init_feq(p, *fl) * (1 + 0.01 * np.random.default_rng(0).standard_normal((19, 7, 9)))
    r, u, w, T = core.fields(p, f)
    d = core.diag(p, f)
    expect = [r.sum(), (r * u).sum(), (r * w).sum(), (r * (T + 0.5 * (u**2 + w**2))).sum(),
              np.abs(w).max(), (0.5 * r * w**2).max(), (0.5 * r * w**2).sum()]
    np.testing.assert_allclose(d, expect, rtol=1e-13)


def test_growth_fit_recovers_exponent():
    # an exact exponential e^{g t} sampled every 10 steps: every estimator returns g
    g, dt, every = 3.7, 1e-5, 10
    t = np.arange(401) * every * dt
    d = np.zeros((401, 7))
    d[:, 4] = 0.01 * np.exp(g * t)
    d[:, 5] = 0.5 * 2.0 * d[:, 4] ** 2
    d[:, 6] = 7.0 * d[:, 4] ** 2
    gu, ge, gk = fit.growth_rates(d, dt, every)
    assert gu == pytest.approx(g, rel=1e-10)
    assert ge == pytest.approx(g, rel=1e-10)
    assert gk == pytest.approx(g, rel=1e-10)
    assert fit.window(401) == slice(101, 401)


def test_mean_density_profile_by_brute_force_and_mass():
    # the averaged density profile (Sec. IV.A): the mean of rho = sum_q f_q
    # along the interface direction x, row by row
    rng = np.random.default_rng(21)
    p = core.Params(nx=13, ny=7, dx=0.01, dy=0.01, dt=1e-5, tau=1e-5)
    f = 0.05 + rng.random((19, p.ny, p.nx))
    md = core.mean_density(p, f)
    brute = np.array([sum(sum(f[q, j, i] for q in range(19)) for i in range(p.nx)) / p.nx for j in range(p.ny)])
    np.testing.assert_allclose(md, brute, rtol=1e-15)
    np.testing.assert_allclose(md, core.fields(p, f)[0].mean(axis=1), rtol=1e-14)
    # nx times its sum is the mass of the state
    assert md.sum() * p.nx == pytest.approx(core.diag(p, f)[0], rel=1e-14)
    # a state uniform along x gives back its rows (to the rounding of nx equal terms over nx)
    g = np.repeat(f[:, :, :1], p.nx, axis=2)
    np.testing.assert_allclose(core.mean_density(p, g), g[:, :, 0].sum(axis=0), rtol=1e-15)


@pytest.mark.parametrize("gamma", [3.0, 9.5])
def test_linear_stage_rate_recovers_a_planted_exponent(gamma):
    # a decay into exp(2 gamma t) that saturates later (the shape of E_max in
    # Sec. IV.A): the fitted rate is the planted one, the window starts 0.05
    # after the minimum and stops once ln E has risen by 4 (before saturation)
    dt = 5e-4
    t = np.arange(2000) * dt
    lnE = np.where(t < 0.1, -6.0 - 30.0 * t, -9.0 + 2.0 * gamma * (t - 0.1))
    lnE = np.minimum(lnE, -2.0)
    g, first, last = fit.linear_stage_rate(np.exp(lnE), dt)
    assert g == pytest.approx(gamma, rel=1e-10)
    assert first == 200 + 100
    assert lnE[last] >= lnE[first] + 4.0 and lnE[last - 1] < lnE[first] + 4.0 and lnE[last] < -2.0
    # a run that ends inside the growth: the window reaches the last sample
    g2, _, last2 = fit.linear_stage_rate(np.exp(lnE[:400]), dt)
    assert g2 == pytest.approx(gamma, rel=1e-10) and last2 == 399
