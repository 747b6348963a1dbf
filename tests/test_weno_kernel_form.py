"""The WENO5 flux as the FP32 kernels write it, checked against the oracle's
flux of Sec. III.A, Eqs. 48-55, in double precision on the CPU.

The kernels rewrite the flux algebraically (their comment in klb_device.cuh
gives the derivation): smoothness indicators scaled by 3/4 (so is epsilon),
the weights over a common denominator (products of the other two squared
indicators), numerator and denominator scaled by 10, and the factor v of
F = v f taken out of the flux by homogeneity, h(v f; eps) = v h(f; eps / v^2).
Each rewrite is exact in real arithmetic, so the rewritten flux, evaluated
here in float64, must equal the oracle's to rounding.  A slip in one of the
constants (11/4, 5/2, -5/4, 5/6, 1/3, 1/2, 6, 3) or in a difference's sign
moves the result far outside that."""
import numpy as np
import pytest

from oracle import core


def kernel_form(a, b, c, d, e, eps34):
    """The flux in the kernels' form; eps34 is 3/4 of the epsilon of Eq. 52
    (divided by v^2 when the stencil holds f rather than F = v f)."""
    d1, d2, d3, e4 = a - b, c - b, d - c, d - e
    s1 = d1 * (d1 + 2.75 * d2) + 2.5 * d2 * d2 + eps34
    s2 = d2 * (d2 - 1.25 * d3) + d3 * d3 + eps34
    s3 = e4 * (e4 + 2.75 * d3) + 2.5 * d3 * d3 + eps34
    p1, p2, p3 = s1 * s1, s2 * s2, s3 * s3
    P23, P13, P12 = p2 * p3, p1 * p3, p1 * p2
    t3 = d3 + d3
    G1 = 5.0 / 6.0 * d2 + 1.0 / 3.0 * d1
    G2 = d2 + t3
    G3 = 0.5 * e4 + t3
    num = G1 * P23 + G2 * P13 + G3 * P12
    den = P23 + 6.0 * P13 + 3.0 * P12
    return c + num / den


def _stencils(rng, n):
    out = []
    for k in range(n):
        F5 = rng.normal(size=5) * 10.0 ** rng.uniform(-3, 1)
        if k % 3 == 0:
            F5[3:] += 5.0 * rng.choice([-1.0, 1.0])  # a jump: weights far from optimal
        if k % 5 == 0:
            F5 = 1.0 + 1e-3 * np.arange(5) ** 2 * rng.uniform(0.5, 2)  # smooth data: weights near optimal
        out.append(F5)
    return out


@pytest.mark.parametrize("eps", [1e-6, 1e-3, 1.0])
def test_kernel_form_equals_the_oracle_flux(eps):
    rng = np.random.default_rng(1010)
    for F5 in _stencils(rng, 300):
        ref = core.weno5_face(F5, eps)
        got = kernel_form(*F5, 0.75 * eps)
        assert got == pytest.approx(ref, rel=1e-11, abs=1e-13 * np.abs(F5).max()), F5


@pytest.mark.parametrize("v", [1.0, 2.0, 3.0, -1.0, -2.0, -3.0])
def test_velocity_factored_out(v):
    # the kernels reconstruct on f with eps / v^2 and multiply by v in the
    # update; the oracle reconstructs F = v f (the reading of Sec. III.A with
    # an absolute epsilon).  Upwind order is the same stencil for both.
    rng = np.random.default_rng(int(10 * v) + 40)
    eps = 1e-6
    for f5 in _stencils(rng, 200):
        ref = core.weno5_face(v * f5, eps)
        got = v * kernel_form(*f5, 0.75 * eps / (v * v))
        assert got == pytest.approx(ref, rel=1e-11, abs=1e-13 * abs(v) * np.abs(f5).max()), (v, f5)


def test_a_wrong_constant_is_caught():
    # the check above is sharp enough to see a single constant off by a little
    rng = np.random.default_rng(7)
    F5s = _stencils(rng, 60)

    def off(a, b, c, d, e, eps34):
        d1, d2, d3, e4 = a - b, c - b, d - c, d - e
        s1 = d1 * (d1 + 2.70 * d2) + 2.5 * d2 * d2 + eps34  # 11/4 mistyped
        s2 = d2 * (d2 - 1.25 * d3) + d3 * d3 + eps34
        s3 = e4 * (e4 + 2.75 * d3) + 2.5 * d3 * d3 + eps34
        p1, p2, p3 = s1 * s1, s2 * s2, s3 * s3
        num = (5 / 6 * d2 + d1 / 3) * p2 * p3 + (d2 + 2 * d3) * p1 * p3 + (0.5 * e4 + 2 * d3) * p1 * p2
        den = p2 * p3 + 6 * p1 * p3 + 3 * p1 * p2
        return c + num / den

    worst = max(abs(off(*F5, 0.75e-6) - core.weno5_face(F5, 1e-6)) / max(np.abs(F5).max(), 1e-30) for F5 in F5s)
    assert worst > 1e-6
