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
