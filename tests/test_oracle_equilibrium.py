"""Pins of the oracle's velocity set, F_k(T) and f^(0) (Sec. II of the paper).

Each check is a closed form or an invariant that the paper states, evaluated by
brute-force sums over the oracle's own tables: a wrong angle, sign, ring index,
coefficient or dropped term in oracle/oklb.c fails at least one of them.
"""
import itertools

import numpy as np
import pytest

from oracle import core

V = (1.0, 2.0, 3.0)


def _ring(q):
    return 0 if q == 0 else 1 + (q - 1) // 6


def test_velocity_geometry():
    # Eq. (5): v_ki = v_k (cos 2 pi i / 6, sin 2 pi i / 6), i = 1..6.
    vx, vy = core.velocity_set(V)
    assert vx[0] == 0.0 and vy[0] == 0.0
    for q in range(1, 19):
        k, i = _ring(q), (q - 1) % 6 + 1
        assert np.hypot(vx[q], vy[q]) == pytest.approx(V[k - 1], rel=1e-15)
        ang = np.arctan2(vy[q], vx[q]) % (2 * np.pi)
        assert ang == pytest.approx((2 * np.pi * i / 6) % (2 * np.pi), abs=1e-14)
    # zero components are exact zeros (they carry no flux)
    assert sum(1 for q in range(19) if vx[q] == 0.0) == 1
    assert sum(1 for q in range(19) if vy[q] == 0.0) == 7


@pytest.mark.parametrize("k", [1, 2, 3])
def test_isotropy(k):
    # Eqs. (7)-(8): sum_i v_a v_b = 3 v_k^2 delta_ab,
    # sum_i v_a v_b v_c v_d = (3/4) v_k^4 Delta_abcd; odd ranks (1, 3, 5) vanish.
    vx, vy = core.velocity_set(V)
    qs = range(1 + 6 * (k - 1), 1 + 6 * k)
    comp = lambda q, a: vx[q] if a == 0 else vy[q]
    d = lambda a, b: 1.0 if a == b else 0.0
    vk = V[k - 1]
    for a, b in itertools.product(range(2), repeat=2):
        s = sum(comp(q, a) * comp(q, b) for q in qs)
        assert s == pytest.approx(3 * vk**2 * d(a, b), abs=1e-13)
    for a, b, c, e in itertools.product(range(2), repeat=4):
        s = sum(comp(q, a) * comp(q, b) * comp(q, c) * comp(q, e) for q in qs)
        Delta = d(a, b) * d(c, e) + d(a, c) * d(b, e) + d(a, e) * d(b, c)
        assert s == pytest.approx(0.75 * vk**4 * Delta, abs=1e-12)
    for rank in (1, 3, 5):
        for idx in itertools.product(range(2), repeat=rank):
            s = sum(np.prod([comp(q, a) for a in idx]) for q in qs)
            assert abs(s) < 1e-12


@pytest.mark.parametrize("T", [0.3, 0.5, 0.8, 1.0, 1.25, 1.5, 2.2])
def test_Fk_requirements(T):
    # Eqs. (40)-(43): sum_ki F_k = 1, sum_k F_k v_k^2 = T/3,
    # sum_k F_k v_k^4 = 4T^2/3, sum_k F_k v_k^6 = 8T^3.
    F = core.Fk(T, V)
    assert F[0] + 6 * (F[1] + F[2] + F[3]) == pytest.approx(1.0, abs=1e-14)
    for power, rhs in ((2, T / 3), (4, 4 * T**2 / 3), (6, 8 * T**3)):
        s = sum(F[k] * V[k - 1] ** power for k in (1, 2, 3))
        assert s == pytest.approx(rhs, rel=1e-13)


def test_Fk_values_and_sign():
    # F_k(T = 1) for v = (1, 2, 3) solves the 4x4 Vandermonde-type system of
    # Eqs. (40)-(43); solve it independently with numpy and compare.
    for T in (1.0, 1.5, 0.4):
        A = np.array([[1.0, 6.0, 6.0, 6.0],
                      [0.0, 1.0, 4.0, 9.0],
                      [0.0, 1.0, 16.0, 81.0],
                      [0.0, 1.0, 64.0, 729.0]])
        b = np.array([1.0, T / 3, 4 * T**2 / 3, 8 * T**3])
        F_ref = np.linalg.solve(A, b)
        np.testing.assert_allclose(core.Fk(T, V), F_ref, rtol=1e-12, atol=1e-15)
    # F_0 is negative at T = 1.5 and must not be clamped
    assert core.Fk(1.5, V)[0] < 0


STATES = [
    (1.0, 0.0, 0.0, 1.0),
    (2.3, 0.31, -0.17, 0.9),
    (0.7, -0.45, 0.2, 1.5),   # F_0 < 0
    (5.0, 0.25, 0.01, 0.3),
    (1.0, 0.5, 0.5, 0.6),
]


@pytest.mark.parametrize("rho,ux,uy,T", STATES)
def test_equilibrium_moments(rho, ux, uy, T):
    # Eq. (10): sum f0 (1, v, (v-u)^2/2) = (rho, rho u, rho T);
    # Eq. (11): sum f0 v_a v_b = P delta_ab + rho u_a u_b;
    # Eq. (12): sum f0 v^2 v_a / 2 = u_a (2P + rho u^2/2), P = rho T.
    vx, vy = core.velocity_set(V)
    f0 = core.feq(rho, ux, uy, T, V)
    P = rho * T
    u = np.array([ux, uy])
    vel = np.stack([vx, vy], axis=1)
    scale = rho * (1 + T + u @ u) ** 2
    tol = 1e-13 * scale
    assert abs(f0.sum() - rho) < tol
    np.testing.assert_allclose(f0 @ vel, rho * u, atol=tol)
    c = vel - u
    assert abs((f0 * 0.5 * (c**2).sum(1)).sum() - rho * T) < tol
    for a, b in itertools.product(range(2), repeat=2):
        lhs = (f0 * vel[:, a] * vel[:, b]).sum()
        rhs = P * (a == b) + rho * u[a] * u[b]
        assert abs(lhs - rhs) < tol
    v2 = (vel**2).sum(1)
    for a in range(2):
        lhs = (f0 * 0.5 * v2 * vel[:, a]).sum()
        rhs = u[a] * (2 * P + 0.5 * rho * (u @ u))
        assert abs(lhs - rhs) < tol


@pytest.mark.parametrize("rho,ux,uy,T", STATES)
def test_moments_roundtrip(rho, ux, uy, T):
    # moments(f0(rho, u, T)) returns (rho, u, T): Eq. (10) read both ways.
    got = core.moments(core.feq(rho, ux, uy, T, V), V)
    np.testing.assert_allclose(got, (rho, ux, uy, T), rtol=1e-13, atol=1e-14)


def test_requirements_FK_long_form():
    # The ten long-form requirements Eqs. (30)-(39) by brute force over the
    # 19 velocities at a random u: each must hold to rounding.
    rng = np.random.default_rng(7)
    vx, vy = core.velocity_set(V)
    vel = np.stack([vx, vy], axis=1)
    v2 = (vel**2).sum(1)
    for T in (0.7, 1.3):
        F = core.Fk(T, V)
        Fq = np.array([F[_ring(q)] for q in range(19)])
        u = rng.uniform(-0.5, 0.5, 2)
        u2 = u @ u
        vu = vel @ u
        d = np.eye(2)
        chk = lambda lhs, rhs: np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-13)
        chk(Fq.sum(), 1.0)                                             # (30)
        chk((Fq * vu**2).sum(), T * u2)                                 # (31)
        chk((Fq[:, None] * vel * vu[:, None]).sum(0), T * u)            # (32)
        chk((Fq[:, None] * vel * (vu**3)[:, None]).sum(0), 3 * T**2 * u2 * u)  # (33)
        chk((Fq * v2 / 2).sum(), T)                                     # (34)
        chk((Fq * v2 / 2 * vu**2).sum(), 2 * T**2 * u2)                 # (35)
        chk(np.einsum("q,qa,qb->ab", Fq, vel, vel), T * d)              # (36)
        chk(np.einsum("q,qa,qb,q->ab", Fq, vel, vel, vu**2), T**2 * (u2 * d + 2 * np.outer(u, u)))  # (37)
        chk((Fq[:, None] * (v2 / 2)[:, None] * vel * vu[:, None]).sum(0), 2 * T**2 * u)  # (38)
        chk((Fq[:, None] * (v2 / 2)[:, None] * vel * (vu**3)[:, None]).sum(0), 9 * T**3 * u2 * u)  # (39)
