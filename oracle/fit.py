"""Growth-rate fit of the Kelvin-Helmholtz runs (Sec. IV of the paper).

TEST INFRASTRUCTURE ONLY.

The paper obtains the growth coefficient gamma from the slope of a straight
line fitted to ln E_x|max(t) over the initial growth stage, with
E_x = rho u^2 / 2 of the cross-stream velocity component, and notes that this
slope is 2 gamma (Sec. IV.A, paragraph before Eq. 66).  The window is not
stated; the reading used here is a fixed window: ordinary least squares over
the last 75% of the samples.
"""
from __future__ import annotations

import numpy as np


def ols_slope(t, y):
    """Least-squares slope of y against t (closed form of the normal equations)."""
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y)
    tm = t.mean()
    return np.sum((t - tm) * (y - y.mean())) / np.sum((t - tm) ** 2)


def window(n_samples: int) -> slice:
    """Indices of the fit window: the last 75% of the samples."""
    start = n_samples - (3 * n_samples) // 4
    return slice(start, n_samples)


def growth_rates(diag, dt: float, sample_every: int):
    """(gamma from ln max|u_y|, gamma from ln max E_x / 2, gamma from ln sum E_x / 2)
    for a diagnostics series diag[m][7] sampled every `sample_every` steps from t=0."""
    d = np.asarray(diag)
    m = d.shape[0]
    t = np.arange(m) * sample_every * dt
    w = window(m)
    g_uy = ols_slope(t[w], np.log(np.real(d[w, 4])))
    g_ex = 0.5 * ols_slope(t[w], np.log(np.real(d[w, 5])))
    g_ke = 0.5 * ols_slope(t[w], np.log(d[w, 6]))
    return g_uy, g_ex, g_ke


def linear_stage_rate(E, dt_sample: float, skip: float = 0.05, rise: float = 4.0):
    """gamma of the initial growth stage of a long run (Sec. IV.A: E_x|max grows
    as exp(2 gamma t) there), with the stage fixed by rule since the paper picks
    it by eye: it starts `skip` time units after the minimum of ln E (where
    the seeded perturbation has decayed into the growing mode) and ends at the
    first sample where ln E has risen by `rise` above its value at the start,
    or at the last sample.  gamma = half the least-squares slope of ln E over
    those samples.  Returns (gamma, first, last) sample indices included."""
    lnE = np.log(np.asarray(E, dtype=np.float64))
    n = len(lnE)
    t = np.arange(n) * dt_sample
    first = min(n - 2, int(np.argmin(lnE)) + int(round(skip / dt_sample)))
    last = first + 1
    while last < n - 1 and lnE[last] < lnE[first] + rise:
        last += 1
    return 0.5 * ols_slope(t[first:last + 1], lnE[first:last + 1]), first, last
