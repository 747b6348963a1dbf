"""The WENO5 flux as the FP32 kernels write it, checked against the oracle's
flux of Sec. III.A, Eqs. 48-55, on the CPU.

The kernels rewrite the flux algebraically (their comment in klb_device.cuh
gives the derivation): smoothness indicators scaled by 3/4 (so is epsilon),
the candidates taken relative to the upwind value c, numerator and
denominator scaled by 10, the weights alpha_q = delta_q / (eps + sigma_q)^2 of
Eq. 52 as reciprocals of the squared indicators, and the factor v of F = v f
taken out of the flux by homogeneity, h(v f; eps) = v h(f; eps / v^2).

1. Each rewrite is exact in real arithmetic, so the rewritten flux, evaluated
   in float64, must equal the oracle's to rounding.  A slip in one of the
   constants (11/4, 5/2, -5/4, 5/6, 1/3, 1/2, 6, 3) or in a difference's sign
   moves the result far outside that.
2. The kernels' FP32 operation order (every multiply, add and fused
   multiply-add rounded to float32, the reciprocal flushing subnormal inputs
   and results to zero as the hardware approximation does) must stay finite
   and within FP32 rounding of the oracle over the range the library accepts:
   epsilon down to 1e-10 and beyond, uniform data, jumps of f up to 1e8.  A
   common denominator of products of the squared indicators (one reciprocal
   per face) spans sigma^4 and fails there; the test shows that too.
"""
import numpy as np
import pytest

from oracle import core


def kernel_form(a, b, c, d, e, eps34):
    """The flux in the kernels' form, in float64; eps34 is 3/4 of the epsilon
    of Eq. 52 (divided by v^2 when the stencil holds f rather than F = v f)."""
    d1, d2, d3, e4 = a - b, c - b, d - c, d - e
    s1 = d1 * (d1 + 2.75 * d2) + 2.5 * d2 * d2 + eps34
    s2 = d2 * (d2 - 1.25 * d3) + d3 * d3 + eps34
    s3 = e4 * (e4 + 2.75 * d3) + 2.5 * d3 * d3 + eps34
    w1, w2, w3 = 1.0 / (s1 * s1), 1.0 / (s2 * s2), 1.0 / (s3 * s3)
    t3 = d3 + d3
    G1 = 5.0 / 6.0 * d2 + 1.0 / 3.0 * d1
    G2 = d2 + t3
    G3 = 0.5 * e4 + t3
    num = G1 * w1 + G2 * w2 + G3 * w3
    den = w1 + 6.0 * w2 + 3.0 * w3
    return c + num / den


# --- float32 model of the kernels' operation order ---------------------------
F32 = np.float32
_TINY = F32(2.0 ** -126)


def _fma(x, y, z):
    # x * y is exact in float64 for float32 inputs; the sum is rounded once to
    # float64 and once to float32 (a model of the single rounding of the fused
    # operation, off by at most one float32 unit in rare halfway cases)
    return F32(np.float64(x) * np.float64(y) + np.float64(z))


def _mul(x, y):
    return F32(F32(x) * F32(y))


def _add(x, y):
    return F32(F32(x) + F32(y))


def _rcp(x):
    """rcp.approx.ftz.f32: subnormal input -> infinity, subnormal result -> 0;
    modelled as the correctly rounded reciprocal otherwise."""
    x = F32(x)
    if abs(x) < _TINY:
        return F32(np.copysign(np.inf, x))
    r = F32(1.0 / np.float64(x))
    return F32(0.0) if abs(r) < _TINY else r


def _indicators_f32(a, b, c, d, e, eps34):
    a, b, c, d, e, eps34 = (F32(v) for v in (a, b, c, d, e, eps34))
    d1, d2, d3, e4 = _fma(b, -1, a), _fma(b, -1, c), _fma(c, -1, d), _fma(e, -1, d)
    a2, a3 = _mul(d2, d2), _mul(d3, d3)
    s1 = _fma(d1, _fma(2.75, d2, d1), _fma(2.5, a2, eps34))
    s2 = _fma(d2, _fma(-1.25, d3, d2), _fma(d3, d3, eps34))
    s3 = _fma(e4, _fma(2.75, d3, e4), _fma(2.5, a3, eps34))
    G1 = _fma(5.0 / 6.0, d2, _mul(1.0 / 3.0, d1))
    t3 = _add(d3, d3)
    return c, (s1, s2, s3), (G1, _add(d2, t3), _fma(0.5, e4, t3))


def kernel_form_f32(a, b, c, d, e, eps34):
    """ArithF32::weno, operation by operation, in float32."""
    with np.errstate(all="ignore"):
        c, (s1, s2, s3), (G1, G2, G3) = _indicators_f32(a, b, c, d, e, eps34)
        r1, r2, r3 = _rcp(s1), _rcp(s2), _rcp(s3)
        w1, w2, w3 = _mul(r1, r1), _mul(r2, r2), _mul(r3, r3)
        num = _fma(G1, w1, _fma(G2, w2, _mul(G3, w3)))
        den = _fma(6.0, w2, _fma(3.0, w3, w1))
        return _fma(num, _rcp(den), c)


def product_form_f32(a, b, c, d, e, eps34):
    """The common denominator of products of the squared indicators (one
    reciprocal per face), in float32: P_23 = s_2^2 s_3^2 etc."""
    with np.errstate(all="ignore"):
        c, (s1, s2, s3), (G1, G2, G3) = _indicators_f32(a, b, c, d, e, eps34)
        p1, p2, p3 = _mul(s1, s1), _mul(s2, s2), _mul(s3, s3)
        P23, P13, P12 = _mul(p2, p3), _mul(p1, p3), _mul(p1, p2)
        num = _fma(G1, P23, _fma(G2, P13, _mul(G3, P12)))
        den = _fma(6.0, P13, _fma(3.0, P12, P23))
        return _fma(num, _rcp(den), c)


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


@pytest.mark.parametrize("eps", [1e-10, 1e-6, 1e-3, 1.0])
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
        w1, w2, w3 = 1 / s1 ** 2, 1 / s2 ** 2, 1 / s3 ** 2
        num = (5 / 6 * d2 + d1 / 3) * w1 + (d2 + 2 * d3) * w2 + (0.5 * e4 + 2 * d3) * w3
        return c + num / (w1 + 6 * w2 + 3 * w3)

    worst = max(abs(off(*F5, 0.75e-6) - core.weno5_face(F5, 1e-6)) / max(np.abs(F5).max(), 1e-30) for F5 in F5s)
    assert worst > 1e-6


def _range_cases():
    """Stencils over the range the library accepts: uniform data, a jump and
    an isolated spike of height J, and random data around J, for J from 1e-4
    to 1e8, each with epsilon 1e-6 (the paper's) and 1e-10."""
    rng = np.random.default_rng(4124)
    out = []
    for eps in (1e-6, 1e-10):
        for J in (1e-4, 1e-3, 1.0, 1e3, 1e4, 1e5, 1e6, 1e8):
            out.append(("uniform", eps, np.full(5, J)))
            out.append(("jump", eps, np.array([0.0, 0.0, 0.0, J, J])))
            out.append(("spike", eps, np.array([0.0, 0.0, 0.0, 0.0, J])))
            out.append(("kink", eps, np.array([J, J, J, 0.5 * J, 0.0])))
            for _ in range(10):
                out.append(("random", eps, J * (1.0 + rng.normal(size=5) * 10.0 ** rng.uniform(-6, 0))))
    return out


def test_fp32_operation_order_over_the_range():
    # error against the oracle on the float32-rounded stencil, relative to the
    # stencil's scale: the rounding of a handful of float32 operations
    for kind, eps, F5 in _range_cases():
        F5 = F5.astype(np.float32).astype(np.float64)
        ref = core.weno5_face(F5, eps)
        got = float(kernel_form_f32(*F5, 0.75 * eps))
        assert np.isfinite(got), (kind, eps, F5)
        assert abs(got - ref) <= 3e-7 * np.abs(F5).max(), (kind, eps, F5, got, ref)


def test_fp32_with_the_velocity_factor_and_small_eps():
    # the kernels' epsilon per plane is 3/4 eps / v_a^2 for the velocity
    # component v_a (1/2 .. 3 for ring speeds 1, 2, 3): the smallest the
    # library accepts (3/4 eps / max(v)^2 = 2e-19) still gives finite fluxes
    # within rounding of the oracle's on uniform data and on jumps
    eps = 2e-19 * 9.0 / 0.75
    for va in (0.5, 1.0, np.sqrt(3.0) / 2, 3.0):
        for F5 in (np.full(5, 1.0), np.array([0.0, 0.0, 0.0, 1.0, 1.0]), np.array([1.0, 2.0, 4.0, 8.0, 16.0])):
            ref = core.weno5_face(va * F5, eps)
            got = va * float(kernel_form_f32(*F5, 0.75 * eps / va ** 2))
            assert np.isfinite(got) and abs(got - ref) <= 3e-7 * va * np.abs(F5).max(), (va, F5, got, ref)


def test_product_form_fails_over_the_range():
    # the previous form of the kernels (a common denominator of products of
    # the squared indicators) overflows or underflows over the same range
    bad = [(kind, eps, F5[-1]) for kind, eps, F5 in _range_cases()
           if not np.isfinite(product_form_f32(*F5.astype(np.float32), 0.75 * eps))]
    kinds = {(k, e) for k, e, _ in bad}
    assert ("uniform", 1e-10) in kinds  # (eps')^4 underflows: 0 * inf
    assert ("jump", 1e-6) in kinds      # sigma^4 of a jump of 1e5 overflows


def grad_form(a, b, c, d, e, eps):
    """The adjoint kernels' gradient of the flux with respect to (a, b, c, d, e)
    (weno5_grad in klb_adjoint.cuh), in float64: partials with respect to the
    differences D1 = a - b, D2 = c - b, D3 = d - c, E4 = d - e of
    h = c + N / D (N = sum G_q w_q, D = w_1 + 6 w_2 + 3 w_3, w_q = 1 / s_q^2),
    mapped back to the five values."""
    e34 = 0.75 * eps
    D1, D2, D3, E4 = a - b, c - b, d - c, d - e
    s1 = D1 * (D1 + 2.75 * D2) + 2.5 * D2 * D2 + e34
    s2 = D2 * (D2 - 1.25 * D3) + D3 * D3 + e34
    s3 = E4 * (E4 + 2.75 * D3) + 2.5 * D3 * D3 + e34
    r1, r2, r3 = 1 / s1, 1 / s2, 1 / s3
    w1, w2, w3 = r1 * r1, r2 * r2, r3 * r3
    G1, G2, G3 = 5 / 6 * D2 + 1 / 3 * D1, D2 + 2 * D3, 2 * D3 + 0.5 * E4
    rD = 1 / (w1 + 6 * w2 + 3 * w3)
    hh = (G1 * w1 + G2 * w2 + G3 * w3) * rD
    o1, o2, o3 = w1 * rD, w2 * rD, w3 * rD
    m = -2 * rD
    b1, b2, b3 = m * (G1 - hh) * w1 * r1, m * (G2 - 6 * hh) * w2 * r2, m * (G3 - 3 * hh) * w3 * r3
    g1 = o1 / 3 + b1 * (2 * D1 + 2.75 * D2)
    g2 = 5 / 6 * o1 + o2 + b1 * (2.75 * D1 + 5 * D2) + b2 * (2 * D2 - 1.25 * D3)
    g3 = 2 * (o2 + o3) + b2 * (2 * D3 - 1.25 * D2) + b3 * (2.75 * E4 + 5 * D3)
    g4 = 0.5 * o3 + b3 * (2 * E4 + 2.75 * D3)
    return c + hh, np.array([g1, -g1 - g2, 1 + g2 - g3, g3 + g4, -g4])


@pytest.mark.parametrize("eps", [1e-6, 1e-3])
def test_adjoint_gradient_form_equals_the_oracle_derivative(eps):
    # the oracle's complex-step derivative of its own flux (Eqs. 48-55) is
    # exact to rounding; the adjoint's difference-form gradient must match it
    rng = np.random.default_rng(48)
    hs = 1e-20
    for F5 in _stencils(rng, 200):
        h, g = grad_form(*F5, eps)
        assert h == pytest.approx(core.weno5_face(F5, eps), rel=1e-11, abs=1e-13 * np.abs(F5).max())
        ref = np.array([np.imag(core.weno5_face(F5 + 1j * hs * np.eye(5)[k], eps, cs=True)) / hs for k in range(5)])
        assert np.abs(g - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max()), (F5, g, ref)
