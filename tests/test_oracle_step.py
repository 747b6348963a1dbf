"""Pins of the oracle's full time step (Sec. III.A, Eq. 47 of the paper).

Invariants and textbook special cases of the forward-Euler / WENO5 / BGK step:
a uniform state is a fixed point; mass, momentum and energy are conserved on a
periodic domain (the flux form telescopes and f^(0) carries the moments of f);
without collisions and with linear weights every velocity plane evolves by the
von Neumann amplification factor of the 5th-order upwind stencil; with a
uniform state the non-equilibrium part decays by exactly (1 - dt/tau) per
step; the step commutes with a mirror reflection in x; y-uniform data stay
y-uniform bitwise; a pressure pulse travels at the sound speed sqrt(2T) of the
gamma = 2 gas the model recovers (Sec. II.B).
"""
import numpy as np
import pytest

from oracle import core
from paper_1010_4124_gb300 import inputs

V = (1.0, 2.0, 3.0)


def _params(nx, ny, dx=0.01, dy=0.01, dt=1e-4, tau=1e-4, bcx="periodic", bcy="periodic", eps=1e-6):
    return core.Params(nx=nx, ny=ny, dx=dx, dy=dy, dt=dt, tau=tau, v=V,
                       bc_x=(bcx, bcx), bc_y=(bcy, bcy), eps=eps)


@pytest.mark.parametrize("bc", ["periodic", "outflow", "fixed_eq"])
def test_uniform_state_is_fixed_point(bc):
    p = _params(12, 10, bcx=bc, bcy=bc)
    shape = (p.ny, p.nx)
    fl = [np.full(shape, v) for v in (1.3, 0.2, -0.1, 0.9)]
    f = core.init_feq(p, *fl)
    fixed = core.fixed_ghosts(p, *fl)
    f1, _ = core.run(p, f, 10, fixed=fixed)
    np.testing.assert_allclose(f1, f, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("seed", [0, 1])
def test_conservation_periodic(seed):
    p = _params(24, 20, dx=0.01, dy=0.015, dt=1e-4, tau=3e-4)
    fl = inputs.smooth_random_fields(p.nx, p.ny, seed, amp=0.1)
    f = core.init_feq(p, *fl)
    # move off equilibrium so that the collision term is active
    f = f * (1.0 + 0.01 * np.random.default_rng(seed).standard_normal(f.shape))
    d0 = core.diag(p, f)
    f1, _ = core.run(p, f, 20)
    d1 = core.diag(p, f1)
    for k in (0, 1, 2, 3):  # mass, momentum x, momentum y, energy
        scale = abs(d0[0]) if k in (1, 2) else abs(d0[k])
        assert abs(d1[k] - d0[k]) <= 20 * 1e-13 * scale, (k, d0[k], d1[k])


def _mode_factor(c_dt_over_d, theta, positive):
    m = np.arange(-2, 3)
    c = np.array([2.0, -13.0, 47.0, 27.0, -3.0]) / 60.0
    if positive:
        S = np.sum(c * (np.exp(1j * m * theta) - np.exp(1j * (m - 1) * theta)))
    else:
        S = np.sum(c * (np.exp(1j * (1 - m) * theta) - np.exp(-1j * m * theta)))
    return c_dt_over_d * S


def test_von_neumann_single_mode():
    # tau -> infinity (no collision), eps -> infinity (linear weights): each
    # plane q is advected by its own velocity, and a Fourier mode is multiplied
    # by G_q = 1 - (dt/dx) v_x S_x - (dt/dy) v_y S_y.
    nx, ny = 16, 12
    p = _params(nx, ny, dx=0.01, dy=0.02, dt=1e-4, tau=1e30, eps=1e30)
    vx, vy = core.velocity_set(V)
    kx, ky = 3, 2
    tx, ty = 2 * np.pi * kx / nx, 2 * np.pi * ky / ny
    I, J = np.meshgrid(np.arange(nx), np.arange(ny))
    phase = np.exp(1j * (tx * I + ty * J))
    f = np.stack([2.0 + np.real(phase)] * 19)
    f1 = core.step(p, f)
    for q in range(19):
        G = 1.0
        if vx[q] != 0:
            G -= _mode_factor(p.dt / p.dx * vx[q], tx, vx[q] > 0)
        if vy[q] != 0:
            G -= _mode_factor(p.dt / p.dy * vy[q], ty, vy[q] > 0)
        expect = 2.0 + np.real(G * phase)
        np.testing.assert_allclose(f1[q], expect, rtol=0, atol=1e-13)


def test_bgk_relaxation_factor():
    # Uniform state: no flux; f - f^(0) shrinks by exactly (1 - dt/tau).
    p = _params(8, 8, dt=3e-5, tau=1e-4)
    vx, vy = core.velocity_set(V)
    rho, ux, uy, T = 1.1, 0.15, -0.05, 0.95
    f0 = core.feq(rho, ux, uy, T, V)
    # a perturbation orthogonal to the collision invariants 1, vx, vy, v^2
    B = np.stack([np.ones(19), vx, vy, vx**2 + vy**2])
    d = np.random.default_rng(1).standard_normal(19)
    d -= B.T @ np.linalg.solve(B @ B.T, B @ d)
    d *= 1e-3
    f = np.broadcast_to((f0 + d)[:, None, None], (19, p.ny, p.nx)).copy()
    f1 = core.step(p, f)
    expect = f0 + (1 - p.dt / p.tau) * d
    np.testing.assert_allclose(f1[:, 3, 4], expect, rtol=0, atol=1e-15)


def test_mirror_reflection_in_x():
    p = _params(20, 14, dx=0.01, dy=0.013, dt=1e-4, tau=2e-4)
    vx, vy = core.velocity_set(V)
    mirror = [int(np.argmin(np.abs(vx + vx[q]) + np.abs(vy - vy[q]))) for q in range(19)]
    fl = inputs.rough_random_fields(p.nx, p.ny, 11)
    f = core.init_feq(p, *fl) * (1 + 0.02 * np.random.default_rng(2).standard_normal((19, p.ny, p.nx)))
    fr = np.empty_like(f)
    for q in range(19):
        fr[mirror[q]] = f[q][:, ::-1]
    a = core.step(p, f)
    b = core.step(p, fr)
    for q in range(19):
        np.testing.assert_allclose(b[mirror[q]][:, ::-1], a[q], rtol=1e-13, atol=1e-14)


def test_y_uniform_stays_bitwise_uniform():
    pb = inputs.sod(nx=60, ny=4, steps=50)
    p = core.Params(nx=pb.nx, ny=pb.ny, dx=pb.dx, dy=pb.dy, dt=pb.dt, tau=pb.tau,
                    bc_x=pb.bc_x, bc_y=pb.bc_y)
    fl = inputs.fields(pb)
    f = core.init_feq(p, *fl)
    f1, _ = core.run(p, f, pb.steps, fixed=core.fixed_ghosts(p, *fl))
    for j in range(1, 4):
        assert np.array_equal(f1[:, j, :], f1[:, 0, :])


def test_sound_speed_gamma2():
    # Small pressure pulse on a uniform gas (rho, T) = (1, 1): two acoustic
    # pulses leave at +-c with c = sqrt(gamma p / rho) = sqrt(2 T).
    nx = 200
    dx = 1.0 / nx
    dt = 0.03 * dx / 3.0
    p = core.Params(nx=nx, ny=1, dx=dx, dy=dx, dt=dt, tau=dt)
    x = (np.arange(nx) + 0.5) * dx
    bump = 1e-3 * np.exp(-((x - 0.5) / 0.04) ** 2)
    rho = (1.0 + bump)[None, :]
    T = np.ones_like(rho)
    z = np.zeros_like(rho)
    f = core.init_feq(p, rho, z, z, T)
    t_end = 0.2
    n = int(round(t_end / dt))
    f1, _ = core.run(p, f, n)
    r, u, w, TT = core.fields(p, f1)
    pres = (r * TT)[0] - 1.0
    right = np.arange(nx // 2 + 10, nx)
    i = right[np.argmax(pres[right])]
    y0, y1, y2 = pres[i - 1], pres[i], pres[i + 1]
    xpk = x[i] + 0.5 * dx * (y0 - y2) / (y0 - 2 * y1 + y2)
    c = (xpk - 0.5) / (n * dt)
    assert c == pytest.approx(np.sqrt(2.0), rel=0.01)


def test_complex_step_tangent_matches_central_fd():
    # The complex build differentiates the step exactly; compare with central
    # finite differences of the real build.
    p = _params(10, 9, dx=0.01, dy=0.012, dt=1e-4, tau=2e-4, bcx="periodic", bcy="outflow")
    fl = inputs.rough_random_fields(p.nx, p.ny, 4)
    f = core.init_feq(p, *fl)
    d = np.random.default_rng(9).standard_normal(f.shape) * 1e-2
    h = 1e-20
    tangent = np.imag(core.step(p, f + 1j * h * d, cs=True)) / h
    e = 1e-6
    fd = (core.step(p, f + e * d) - core.step(p, f - e * d)) / (2 * e)
    np.testing.assert_allclose(tangent, fd, rtol=0, atol=1e-8 * np.abs(tangent).max())


@pytest.mark.parametrize("axis", ["x", "y"])
@pytest.mark.parametrize("bc", ["outflow", "fixed_eq"])
def test_ghost_nodes_by_explicit_padding(axis, bc):
    # Eqs. (57), (63)-(64): one step with `bc` on one axis equals one step on
    # an explicitly padded periodic domain whose three extra layers per side
    # hold the ghost values by definition (copies of the edge node for
    # outflow, f^(0) of the edge node's initial state for fixed_eq).
    nx, ny = 14, 12
    fl = inputs.rough_random_fields(nx, ny, 21)
    bcx = bc if axis == "x" else "periodic"
    bcy = bc if axis == "y" else "periodic"
    p = _params(nx, ny, dx=0.01, dy=0.012, dt=1e-4, tau=2e-4, bcx=bcx, bcy=bcy)
    f = core.init_feq(p, *fl) * (1 + 0.02 * np.random.default_rng(5).standard_normal((19, ny, nx)))
    fixed = core.fixed_ghosts(p, *fl)
    got = core.step(p, f, fixed=fixed)
    ax = 2 if axis == "x" else 1
    n = nx if axis == "x" else ny
    lo_edge = np.take(f, [0], axis=ax)
    hi_edge = np.take(f, [n - 1], axis=ax)
    if bc == "fixed_eq":
        other = ny if axis == "x" else nx
        base = 0 if axis == "x" else 2 * 19 * ny
        lo = fixed[base: base + 19 * other].reshape(19, other)
        hi = fixed[base + 19 * other: base + 2 * 19 * other].reshape(19, other)
        lo_edge = np.expand_dims(lo, ax)
        hi_edge = np.expand_dims(hi, ax)
    padded = np.concatenate([lo_edge] * 3 + [f] + [hi_edge] * 3, axis=ax)
    pp = _params(nx + 6 if axis == "x" else nx, ny + 6 if axis == "y" else ny,
                 dx=0.01, dy=0.012, dt=1e-4, tau=2e-4)
    ref = core.step(pp, padded)
    ref = np.take(ref, np.arange(3, 3 + n), axis=ax)
    np.testing.assert_allclose(got, ref, rtol=1e-14, atol=1e-15)


def test_wrapper_refuses_arrays_of_the_wrong_shape():
    # the C code reads exactly the parameters' sizes: a mismatch is refused
    # before the call instead of being read past
    p = core.Params(nx=6, ny=5, dx=0.01, dy=0.01, dt=1e-4, tau=1e-4)
    good = [np.ones((5, 6)) for _ in range(4)]
    f = core.init_feq(p, *good)
    with pytest.raises(ValueError):
        core.init_feq(p, np.ones((4, 6)), *good[1:])
    with pytest.raises(ValueError):
        core.step(p, f[:, :4])
    with pytest.raises(ValueError):
        core.run(p, f, 1, fixed=np.zeros(5))
    for fn in (core.fields, core.diag, core.mean_density):
        with pytest.raises(ValueError):
            fn(p, f[:18])
