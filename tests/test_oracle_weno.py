"""Pins of the oracle's WENO5 flux (Sec. III.A, Eqs. 48-55 of the paper).

The paper cites Jiang & Shu (J. Comput. Phys. 126, 202, 1996) for the scheme.
The checks below rebuild the scheme from its definitions with numpy linear
algebra -- candidate fluxes as values of the quadratics whose cell averages
match the data on each 3-cell stencil, smoothness indicators as the
sum over l = 1, 2 of the integrals of the squared l-th derivatives of those
quadratics over the cell, optimal weights as the combination that reproduces
the quartic through all five cells -- and compare the oracle with them.
Further: the textbook 5th-order upwind flux, polynomial exactness, observed
order of convergence, and odd symmetry.
"""
import numpy as np
import pytest
from numpy.polynomial import polynomial as P

from oracle import core


def _cell_avg_matrix(cells, degree):
    """M[r, m] = average of x^m over the unit cell centred at cells[r]."""
    M = np.zeros((len(cells), degree + 1))
    for r, j in enumerate(cells):
        for m in range(degree + 1):
            M[r, m] = ((j + 0.5) ** (m + 1) - (j - 0.5) ** (m + 1)) / (m + 1)
    return M


STENCILS = ([-2, -1, 0], [-1, 0, 1], [0, 1, 2])


def _quadratic(F5, s):
    cells = STENCILS[s]
    vals = np.array([F5[j + 2] for j in cells])
    return np.linalg.solve(_cell_avg_matrix(cells, 2), vals)


def _definition_flux(F5, eps):
    """h_{I+1/2} rebuilt from the Jiang-Shu definitions (cells of unit width, I = 0)."""
    h, beta = [], []
    for s in range(3):
        c = _quadratic(F5, s)
        h.append(P.polyval(0.5, c))
        b = 0.0
        for l in (1, 2):
            d = P.polyder(c, l)
            sq = P.polyint(P.polymul(d, d))
            b += P.polyval(0.5, sq) - P.polyval(-0.5, sq)
        beta.append(b)
    # optimal weights: the delta with sum_q delta_q h_q = quartic value at 1/2
    # for every data vector; solve on the 5 unit vectors (least squares).
    Q = np.linalg.inv(_cell_avg_matrix([-2, -1, 0, 1, 2], 4))
    quart_row = P.polyval(0.5, np.eye(5)).T @ Q  # value at 1/2 of the quartic through e_r
    H = np.zeros((5, 3))
    for r in range(5):
        e = np.zeros(5)
        e[r] = 1.0
        for s in range(3):
            H[r, s] = P.polyval(0.5, _quadratic(e, s))
    delta, *_ = np.linalg.lstsq(H, quart_row, rcond=None)
    a = np.array([delta[s] / (eps + beta[s]) ** 2 for s in range(3)])
    w = a / a.sum()
    return float(w @ np.array(h)), delta, np.array(beta)


def test_optimal_weights_from_definition():
    _, delta, _ = _definition_flux(np.zeros(5), 1e-6)
    np.testing.assert_allclose(delta, [0.1, 0.6, 0.3], atol=1e-13)


def test_smoothness_indicators_from_definition():
    # For a step F = (0,0,0,1,1) the definition gives beta = (0, 4/3, 10/3).
    _, _, beta = _definition_flux(np.array([0.0, 0.0, 0.0, 1.0, 1.0]), 1e-6)
    np.testing.assert_allclose(beta, [0.0, 4.0 / 3.0, 10.0 / 3.0], atol=1e-13)


@pytest.mark.parametrize("seed", range(12))
def test_flux_matches_definition(seed):
    rng = np.random.default_rng(seed)
    F5 = rng.normal(size=5) * 10.0 ** rng.uniform(-3, 1)
    if seed % 3 == 0:
        F5[3:] += 5.0  # a jump: weights far from optimal
    for eps in (1e-6, 1e-2):
        ref, _, _ = _definition_flux(F5, eps)
        got = core.weno5_face(F5, eps)
        assert got == pytest.approx(ref, rel=1e-12, abs=1e-14 * np.abs(F5).max())


def test_linear_weights_is_textbook_upwind5():
    # eps -> infinity: the flux becomes (2, -13, 47, 27, -3)/60 . F_{I-2..I+2}.
    rng = np.random.default_rng(3)
    c = np.array([2.0, -13.0, 47.0, 27.0, -3.0]) / 60.0
    for _ in range(10):
        F5 = rng.normal(size=5)
        assert core.weno5_face(F5, 1e30) == pytest.approx(c @ F5, rel=1e-14, abs=1e-15)


def test_odd_symmetry():
    rng = np.random.default_rng(5)
    for _ in range(10):
        F5 = rng.normal(size=5)
        assert core.weno5_face(-F5, 1e-6) == -core.weno5_face(F5, 1e-6)


def _divergence(F, eps):
    n = F.size
    h = np.array([core.weno5_face(np.take(F, np.arange(i - 2, i + 3), mode="wrap"), eps) for i in range(n)])
    return h - np.roll(h, 1)  # (h_{I+1/2} - h_{I-1/2}) for cells of unit width


@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4])
def test_polynomial_exactness_linear_weights(deg):
    # With linear weights the flux difference reproduces d/dx of point values of
    # polynomials of degree <= 4 exactly (the quartic reconstruction is exact).
    x = np.arange(-10, 11, dtype=np.float64)
    coef = np.arange(1, deg + 2, dtype=np.float64) / 7.0
    # F as point values of p; the face flux reconstructs the function whose
    # cell averages are these point values, so the difference equals p'(x_I).
    F = P.polyval(x, coef)
    dp = P.polyval(x, P.polyder(coef)) if deg > 0 else np.zeros_like(x)
    for I in range(3, len(x) - 3):
        hp = core.weno5_face(F[I - 2:I + 3], 1e30)
        hm = core.weno5_face(F[I - 3:I + 2], 1e30)
        assert hp - hm == pytest.approx(dp[I], abs=1e-9 * (1 + abs(F).max()))


@pytest.mark.parametrize("eps,min_order", [(1e30, 4.9), (1e-6, 4.7)])
def test_convergence_order(eps, min_order):
    # Smooth periodic data F = 1 + 0.1 sin(2 pi x): the flux difference / dx
    # converges to F'(x) at 5th order.
    errs = []
    Ns = [32, 64, 128, 256, 512, 1024]
    for N in Ns:
        x = np.arange(N) / N
        F = 1.0 + 0.1 * np.sin(2 * np.pi * x)
        d = _divergence(F, eps) * N
        errs.append(np.abs(d - 0.2 * np.pi * np.cos(2 * np.pi * x)).mean())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-2] >= min_order, (errs, orders)
    if eps > 1:
        assert abs(orders[-2] - 5.0) < 0.1
