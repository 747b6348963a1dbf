"""The lower-order convection schemes the paper compares with WENO5 (Sec. III.B,
Fig. 2): first-order upwind, second-order upwind and second-order TVD
(minmod).  The paper names them without formulas; the oracle takes the
textbook forms on WENO5's upwind-ordered stencil (c = F_I the upwind node,
b = F_{I-1}, d = F_{I+1}).  Pinned here by what the mathematics fixes -- the
exact derivative of low-degree polynomials, the observed order on smooth data,
the total-variation behaviour on a square wave -- and by the paper's own
statement on the Sod tube: the higher the order, the fewer cells across the
shock; first-order upwind smears, second-order upwind oscillates, TVD does not.
"""
import numpy as np
import pytest

from oracle import core, riemann
from paper_1010_4124_gb300 import inputs

LOW = ("upwind1", "upwind2", "tvd")
LEFT, RIGHT = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)


def face(scheme, st):
    return core.face_flux(scheme, np.asarray(st, dtype=float))


def line_divergence(scheme, F, dx):
    """(h_{i+1/2} - h_{i-1/2}) / dx on a periodic line, v > 0: the face left of
    node i takes the stencil i-3 .. i+1 (upwind node i-1)."""
    N = len(F)
    h = np.array([face(scheme, [F[(i + k) % N] for k in (-3, -2, -1, 0, 1)]) for i in range(N)])
    return (np.roll(h, -1) - h) / dx


@pytest.mark.parametrize("scheme", ("weno5",) + LOW)
def test_constant_data_give_the_constant_flux(scheme):
    for v in (0.0, 1.0, -2.5, 1e-3):
        if scheme == "weno5":  # its candidate coefficients sum to one only up to rounding
            assert face(scheme, [v] * 5) == pytest.approx(v, rel=4e-16)
        else:
            assert face(scheme, [v] * 5) == v


def test_polynomial_data_closed_forms():
    h = 0.01
    for x in (0.3, 0.7, 1.9):
        nodes = x + h * np.arange(-3, 2)  # x_{i-3} .. x_{i+1}; faces h_{i-1/2} (upwind i-1), h_{i+1/2} (upwind i)
        for deg, f, df in ((1, lambda t: 2 * t - 1, lambda t: 2.0), (2, lambda t: t * t, lambda t: 2 * t),
                           (3, lambda t: t**3, lambda t: 3 * t * t)):
            ext = x + h * np.arange(-4, 3)
            F = f(ext)
            hl = {s: face(s, F[0:5]) for s in LOW}   # stencil x_{i-4}..x_i: face between i-2 and i-1... upwind x_{i-2}
            hr = {s: face(s, F[1:6]) for s in LOW}   # upwind node x_{i-1}
            # the divergence at node x_{i-1} (upwind nodes x_{i-2} and x_{i-1} of its two faces)
            xi = x - h
            D = {s: (hr[s] - hl[s]) / h for s in LOW}
            # first-order upwind: (F_i - F_{i-1}) / h; exact for linear data, x^2 -> 2x - h
            if deg == 1:
                assert D["upwind1"] == pytest.approx(df(xi), rel=1e-12)
            if deg == 2:
                assert D["upwind1"] == pytest.approx(2 * xi - h, rel=1e-10)
            # second-order upwind: (3F_i - 4F_{i-1} + F_{i-2}) / (2h); exact up to degree 2, x^3 -> 3x^2 - 2h^2
            if deg <= 2:
                assert D["upwind2"] == pytest.approx(df(xi), rel=1e-10)
            else:
                assert D["upwind2"] == pytest.approx(3 * xi * xi - 2 * h * h, rel=1e-9)
            # TVD on convex increasing data takes the smaller, left difference: it equals second-order upwind
            if deg in (2, 3):
                assert D["tvd"] == pytest.approx(D["upwind2"], rel=1e-12)


def test_tvd_flux_is_first_order_at_an_extremum():
    # b < c > d: the one-sided differences disagree in sign, minmod = 0, h = c
    assert face("tvd", [0.0, 1.0, 3.0, 2.0, 0.0]) == 3.0
    assert face("tvd", [5.0, 4.0, 1.0, 2.0, 9.0]) == 1.0
    # monotone data: the smaller difference, with its sign
    assert face("tvd", [0.0, 1.0, 2.0, 6.0, 7.0]) == 2.5
    assert face("tvd", [9.0, 8.0, 2.0, 1.0, 0.0]) == 1.5


@pytest.mark.parametrize("scheme,lo,hi", [("upwind1", 0.95, 1.05), ("upwind2", 1.95, 2.05), ("tvd", 1.5, 2.1)])
def test_observed_order_on_smooth_periodic_data(scheme, lo, hi):
    errs = []
    Ns = (64, 128, 256)
    for N in Ns:
        x = np.arange(N) / N
        F = 1.0 + 0.1 * np.sin(2 * np.pi * x)
        D = line_divergence(scheme, F, 1.0 / N)
        # the divergence approximates dF/dx at the node
        errs.append(np.abs(D - 0.2 * np.pi * np.cos(2 * np.pi * x)).mean())
    order = np.log2(errs[-2] / errs[-1])
    assert lo <= order <= hi, (errs, order)


def _advect_square_wave(scheme, steps=40, N=80, cfl=0.4):
    x = np.arange(N) / N
    F = np.where((x > 0.25) & (x < 0.55), 1.0, 0.0)
    tv = [np.abs(np.diff(np.append(F, F[0]))).sum()]
    for _ in range(steps):
        F = F - cfl * line_divergence(scheme, F, 1.0)
        tv.append(np.abs(np.diff(np.append(F, F[0]))).sum())
    return F, np.array(tv)


def test_total_variation_on_a_square_wave():
    # forward Euler at CFL 0.4: first-order upwind and the minmod scheme do not
    # increase the total variation; second-order upwind does (new extrema)
    for s in ("upwind1", "tvd"):
        F, tv = _advect_square_wave(s)
        assert np.all(np.diff(tv) <= 1e-12), (s, tv)
        assert F.min() >= -1e-14 and F.max() <= 1 + 1e-14
    F, tv = _advect_square_wave("upwind2")
    assert tv[-1] > tv[0] + 0.1
    assert F.min() < -0.01 or F.max() > 1.01


@pytest.mark.parametrize("scheme", LOW)
def test_mirror_reflection_of_the_step(scheme):
    # reflecting the state in x maps the step onto itself for every scheme
    # (the mirrored stencil of a negative velocity component is the reflection;
    # the moment sums run over the velocities in another order, hence rounding)
    rng = np.random.default_rng(3)
    nx, ny = 12, 7
    p = core.Params(nx=nx, ny=ny, dx=0.01, dy=0.01, dt=2e-4, tau=2e-4, scheme=scheme)
    rho = 1.0 + 0.2 * rng.random((ny, nx))
    ux, uy = 0.1 * rng.standard_normal((ny, nx)), 0.1 * rng.standard_normal((ny, nx))
    T = 0.8 + 0.3 * rng.random((ny, nx))
    f = core.init_feq(p, rho, ux, uy, T) * (1 + 0.01 * rng.standard_normal((19, ny, nx)))
    vx, vy = core.velocity_set(p.v)
    # velocity q reflected in x: the q' with (vx, vy) -> (-vx, vy)
    perm = [int(np.argmin(np.abs(vx + vx[q]) + np.abs(vy - vy[q]))) for q in range(19)]
    fr = f[perm][:, :, ::-1].copy()
    g = core.step(p, f)
    gr = core.step(p, fr)
    np.testing.assert_allclose(gr, g[perm][:, :, ::-1], rtol=1e-13, atol=1e-14)


def _sod(scheme, steps=None):
    pb = inputs.sod(nx=200, ny=4)
    p = core.Params(nx=pb.nx, ny=pb.ny, dx=pb.dx, dy=pb.dy, dt=pb.dt, tau=pb.tau, bc_x=pb.bc_x, bc_y=pb.bc_y,
                    scheme=scheme)
    fl = inputs.fields(pb)
    f, _ = core.run(p, core.init_feq(p, *fl), pb.steps if steps is None else steps,
                    fixed=core.fixed_ghosts(p, *fl))
    r, u, w, T = (a[0] for a in core.fields(p, f))
    return (np.arange(pb.nx) + 0.5) * pb.dx, r, r * T, pb


def _shock_width(x, pr, t, dx):
    p_s = riemann.star_state(LEFT, RIGHT, gamma=2.0)[0]
    S = riemann.wave_speeds(LEFT, RIGHT, gamma=2.0)[3]
    lo, hi = 0.1 + 0.1 * (p_s - 0.1), 0.1 + 0.9 * (p_s - 0.1)
    sel = (x > 0.5 + S * t - 0.1) & (x < 0.5 + S * t + 0.1)
    xx, pp = x[sel], pr[sel]

    def crossing(level):
        i = np.where((pp[:-1] >= level) & (pp[1:] < level))[0][-1]
        return xx[i] + dx * (pp[i] - level) / (pp[i] - pp[i + 1])

    return (crossing(lo) - crossing(hi)) / dx


@pytest.fixture(scope="module")
def sod_schemes():
    return {s: _sod(s) for s in ("weno5", "upwind1", "tvd")}


def test_sod_shock_is_narrower_with_higher_order(sod_schemes):
    # Fig. 2: first-order upwind spreads the shock widely, the TVD scheme less,
    # WENO5 over about three to four cells or fewer
    w = {}
    for s, (x, r, pr, pb) in sod_schemes.items():
        w[s] = _shock_width(x, pr, pb.steps * pb.dt, pb.dx)
    assert w["upwind1"] > 5.0, w
    assert w["weno5"] < w["tvd"] < w["upwind1"], w
    assert w["weno5"] <= 4.0, w


def test_sod_oscillations_by_scheme(sod_schemes):
    # the exact density decreases monotonically from 1 to 0.125: total
    # variation 0.875.  First-order upwind and TVD keep it; WENO5 exceeds it
    # by little; second-order upwind oscillates (the textbook form diverges
    # later in the run, see the readings: checked here at 1000 steps)
    tv = {s: np.abs(np.diff(r)).sum() for s, (x, r, pr, pb) in sod_schemes.items()}
    assert tv["upwind1"] == pytest.approx(0.875, abs=1e-3), tv
    assert tv["tvd"] == pytest.approx(0.875, abs=2e-3), tv
    assert tv["weno5"] < 0.875 + 0.03, tv
    x, r, pr, pb = _sod("upwind2", steps=1000)
    assert np.abs(np.diff(r)).sum() > 0.875 + 0.1
