"""The growth-rate fit of the sweep driver (paper_1010_4124_gb300.sweeps), on
synthetic series whose rate is known: an initial decay into an exponential
growth exp(2 gamma t) that later saturates (the shape of E_max in Sec. IV.A)."""
import numpy as np
import pytest

from paper_1010_4124_gb300 import sweeps


def _series(gamma, dt=5e-4, n=800, t_turn=0.08, sat=-1.0, noise=0.0, seed=0):
    t = np.arange(n) * dt
    lnE = np.where(t < t_turn, -7.0 - 20.0 * t, -7.0 - 20.0 * t_turn + 2 * gamma * (t - t_turn))
    lnE = np.minimum(lnE, sat)  # saturation
    lnE = lnE + noise * np.random.default_rng(seed).standard_normal(n)
    return np.exp(lnE), dt


@pytest.mark.parametrize("gamma", [2.0, 5.0, 12.0])
def test_recovers_the_rate_of_an_exponential_stage(gamma):
    E, dt = _series(gamma)
    g, a, b = sweeps.growth_rate(E, dt)
    assert g == pytest.approx(gamma, rel=1e-10)
    # the window starts after the minimum and stops before saturation
    assert a * dt >= 0.08 + 0.05 - dt and np.log(E[b]) < -1.0


def test_noise_averages_out():
    E, dt = _series(8.0, noise=0.05, seed=4)
    g, a, b = sweeps.growth_rate(E, dt)
    assert g == pytest.approx(8.0, rel=0.03)


def test_fitted_laws_recover_their_coefficients():
    res = [{"Dv": d, "gamma": float(np.exp(2.7 - 0.07 * d))} for d in (2, 4, 8, 16)]
    a, b = sweeps.fit_velocity_law(res)
    assert a == pytest.approx(2.7, rel=1e-12) and b == pytest.approx(0.07, rel=1e-10)
    res = [{"Drho": d, "gamma": 5.28 + 0.62 * np.log(d)} for d in (1, 2, 3, 5, 8)]
    c, e = sweeps.fit_density_law(res)
    assert c == pytest.approx(5.28, rel=1e-12) and e == pytest.approx(0.62, rel=1e-10)
