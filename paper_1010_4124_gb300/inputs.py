"""Seeded synthetic workloads of the FDLB step (arXiv:1010.4124).

This module holds only input generation: grids, initial macroscopic fields and
the run parameters of the five workloads.  It contains none of the method's
arithmetic (no equilibrium, no moments, no fluxes), so that both the CUDA path
and the CPU oracle can take their inputs from it.  Every function works on
complex inputs as well (numpy's tanh/sin/exp accept them), which the
complex-step tangent tests use to differentiate through D_v and D_rho.

Workloads (macroscopic initial states; f starts at f^(0) of these fields):
  sod      Sec. III.B, Eq. (56): Sod tube on [0,1], (rho,u,v,T) = (1,0,0,1) for
           x <= 0.5 and (0.125,0,0,0.8) for x > 0.5; nodes at x_i = (i+1/2) dx.
  khi      Kelvin-Helmholtz shear layer, interface along x at y = 0, periodic in
           x and outflow in y: u_x = (u0/2) tanh(y/D_v), rho = (rho1+rho2)/2 +
           (rho1-rho2)/2 tanh(y/D_rho), uniform p, T = p/rho, perturbation
           u_y = a sin(2 pi x/Lx) exp(-(y/(0.05 Ly))^2).  D_v, D_rho in cells.
           Nodes at x_i = i dx, y_j = (j - ny/2 + 1/2) dy.  The shape follows
           the paper's tanh profiles (Eqs. 59-61) rotated so that the shear
           layer lies along the x (fastest, periodic) axis.
  khi4     khi with four sinusoidal modes of seeded random phase (4096^2 case).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

SWEEP_SEED = 1010412
ROOFLINE_PHASE_SEED = 4096
SWEEP_SIZES = ((256, 256), (512, 256), (512, 512), (1024, 512))  # (nx, ny)
SWEEP_DV = (2, 4, 6, 8, 10, 12, 14, 16)
SWEEP_DRHO = (2, 6, 12, 24)


@dataclass
class Problem:
    """Run parameters (grid, spacing, time step, relaxation time, ring speeds,
    boundary kinds) plus the initial-field recipe."""
    name: str
    nx: int
    ny: int
    dx: float
    dy: float
    dt: float
    tau: float
    steps: int
    v: tuple = (1.0, 2.0, 3.0)
    bc_x: tuple = ("periodic", "periodic")
    bc_y: tuple = ("periodic", "periodic")
    sample_every: int = 0
    # KHI recipe
    Dv: float = 4.0
    Drho: float = 4.0
    rho1: float = 5.0
    rho2: float = 1.0
    u0: float = 0.5
    p0: float = 1.5
    amp: float = 0.01
    modes: int = 1
    phase_seed: int | None = None
    envelope: str = "gauss"  # cross-stream envelope of u_y: "gauss" exp(-(y/(0.05 Ly))^2), "exp" exp(-k|y|)

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)


def sod(nx: int = 200, ny: int = 4, steps: int = 5000, dt: float | None = None, tau: float | None = None) -> Problem:
    """Sod tube: domain [0,1] x ny cells, dx = dy = 1/nx, dt = 2e-5 at nx = 200
    (CFL 3 dt/dx = 0.012 kept fixed under refinement), tau = dt."""
    dx = 1.0 / nx
    if dt is None:
        dt = 2e-5 * (200.0 / nx)
    if tau is None:
        tau = dt
    return Problem("sod", nx, ny, dx, dx, dt, tau, steps,
                   bc_x=("fixed_eq", "fixed_eq"), bc_y=("periodic", "periodic"))


def khi(nx: int = 512, ny: int = 512, steps: int = 4000, Dv: float = 4.0, Drho: float = 4.0,
        modes: int = 1, phase_seed: int | None = None, sample_every: int = 10) -> Problem:
    """KHI shear layer: dx = dy = 0.002, dt = tau = 1e-5, rho1 = 5, rho2 = 1,
    u0 = 0.5, p = 1.5, perturbation amplitude 0.01 (one mode) or 0.0025 per
    mode (four modes)."""
    amp = 0.01 if modes == 1 else 0.0025
    return Problem("khi", nx, ny, 0.002, 0.002, 1e-5, 1e-5, steps,
                   bc_x=("periodic", "periodic"), bc_y=("outflow", "outflow"),
                   sample_every=sample_every, Dv=Dv, Drho=Drho, amp=amp, modes=modes,
                   phase_seed=phase_seed)


def roofline_4096(steps: int = 1000) -> Problem:
    """The 4096 x 4096 KHI: D_v = D_rho = 16 cells, four modes of seeded phase."""
    return khi(4096, 4096, steps, Dv=16.0, Drho=16.0, modes=4, phase_seed=ROOFLINE_PHASE_SEED)


def paper_khi(Dv: float, Drho: float, state: str = "A", steps: int = 40000, sample_every: int = 50) -> Problem:
    """The paper's Kelvin-Helmholtz set-ups (Sec. IV) in this library's
    orientation (the interface along x, periodic; the cross-stream direction y,
    outflow).  Domain 0.2 (periodic, the paper's height) x 0.6 (cross-stream,
    the paper's length); dt = tau = 1e-5; perturbation
    u_y = 0.02 sin(k x) exp(-k |y|), k = 10 pi (one wavelength over the
    periodic length).  D_v, D_rho in cells.
      state "A" (Sec. IV.A, the velocity-gradient study): rho 5.0 / 2.0,
        u_x +-0.5, p = 2.5, dx = dy = 0.001 (200 x 600 cells);
      state "B" (Sec. IV.B, the density-gradient study, and the hybrid
        R = D_rho / D_v study of Sec. IV.C): rho 5.0 / 1.25, u_x +-0.5,
        p = 1.5, dx = dy = 0.002 (100 x 300 cells)."""
    if state == "A":
        nx, ny, d, rho2, p0 = 200, 600, 0.001, 2.0, 2.5
    elif state == "B":
        nx, ny, d, rho2, p0 = 100, 300, 0.002, 1.25, 1.5
    else:
        raise ValueError(f"unknown state {state}")
    return Problem(f"khi-{state}", nx, ny, d, d, 1e-5, 1e-5, steps, bc_x=("periodic", "periodic"),
                   bc_y=("outflow", "outflow"), sample_every=sample_every, Dv=float(Dv), Drho=float(Drho),
                   rho1=5.0, rho2=rho2, u0=1.0, p0=p0, amp=0.02, modes=1, envelope="exp")


def sweep_instances(steps: int = 2000, seed: int = SWEEP_SEED):
    """The 32 (D_v, D_rho) instances of the batched sweep, row-major over D_v
    then D_rho, each on a grid size drawn from SWEEP_SIZES by the seed."""
    rng = np.random.default_rng(seed)
    out = []
    for Dv in SWEEP_DV:
        for Dr in SWEEP_DRHO:
            nx, ny = SWEEP_SIZES[int(rng.integers(0, len(SWEEP_SIZES)))]
            out.append(khi(nx, ny, steps, Dv=float(Dv), Drho=float(Dr)))
    return out


def coords(pb: Problem):
    """Node coordinates (X, Y) as [ny][nx] arrays."""
    if pb.name == "sod":
        x = (np.arange(pb.nx) + 0.5) * pb.dx
        y = (np.arange(pb.ny) + 0.5) * pb.dy
    else:
        x = np.arange(pb.nx) * pb.dx
        y = (np.arange(pb.ny) - pb.ny / 2 + 0.5) * pb.dy
    return np.meshgrid(x, y)


def phases(pb: Problem):
    if pb.modes == 1:
        return np.zeros(1)
    rng = np.random.default_rng(pb.phase_seed)
    return rng.uniform(0.0, 2.0 * np.pi, pb.modes)


def perturbation_shape(pb: Problem):
    """u_y of the initial state (the field the adjoint differentiates against)."""
    X, Y = coords(pb)
    Lx, Ly = pb.nx * pb.dx, pb.ny * pb.dy
    if pb.envelope == "exp":  # exp(-k |y|) with k = 2 pi / Lx, the wave number of the first mode
        env = np.exp(-(2.0 * np.pi / Lx) * np.abs(Y))
    else:
        env = np.exp(-(Y / (0.05 * Ly)) ** 2)
    uy = np.zeros_like(X)
    for m, ph in enumerate(phases(pb), start=1):
        uy = uy + pb.amp * np.sin(2.0 * np.pi * m * X / Lx + ph) * env
    return uy


def fields(pb: Problem, Dv=None, Drho=None, uy=None):
    """Initial (rho, ux, uy, T) as [ny][nx] arrays.  Dv / Drho (cells) and the
    u_y field may be overridden (complex values allowed)."""
    X, Y = coords(pb)
    if pb.name == "sod":
        left = X < 0.5
        rho = np.where(left, 1.0, 0.125)
        T = np.where(left, 1.0, 0.8)
        z = np.zeros_like(X)
        return rho, z.copy(), z.copy(), T
    Dv = pb.Dv if Dv is None else Dv
    Drho = pb.Drho if Drho is None else Drho
    ux = 0.5 * pb.u0 * np.tanh(Y / (Dv * pb.dy))
    rho = 0.5 * (pb.rho1 + pb.rho2) + 0.5 * (pb.rho1 - pb.rho2) * np.tanh(Y / (Drho * pb.dy))
    T = pb.p0 / rho
    if uy is None:
        uy = perturbation_shape(pb)
    return rho, ux, np.asarray(uy) + 0.0 * ux, T


def smooth_random_fields(nx: int, ny: int, seed: int, amp: float = 0.05):
    """Smooth periodic random state for parity and conservation tests: a few
    low Fourier modes of seeded random amplitude and phase around
    (rho, ux, uy, T) = (1, 0.1, -0.05, 1)."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx) / nx
    y = np.arange(ny) / ny
    X, Y = np.meshgrid(x, y)
    out = []
    for base in (1.0, 0.1, -0.05, 1.0):
        g = np.full_like(X, base)
        for _ in range(3):
            kx, ky = rng.integers(0, 3, size=2)
            a, ph = rng.uniform(-amp, amp), rng.uniform(0, 2 * np.pi)
            g = g + a * np.sin(2 * np.pi * (kx * X + ky * Y) + ph)
        out.append(g)
    return tuple(out)


def rough_random_fields(nx: int, ny: int, seed: int):
    """Non-smooth state (random jumps) that exercises the nonlinear WENO weights."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 1.5, size=(ny, nx))
    ux = rng.uniform(-0.2, 0.2, size=(ny, nx))
    uy = rng.uniform(-0.2, 0.2, size=(ny, nx))
    T = rng.uniform(0.6, 1.2, size=(ny, nx))
    return rho, ux, uy, T


def blocky_fields(nx: int, ny: int, seed: int, block: int = 8):
    """Piecewise-constant state: uniform blocks of block x block nodes with
    seeded random (rho, ux, uy, T) each, so that most stencils see uniform
    data (smoothness indicators equal to epsilon) and the rest a jump."""
    rng = np.random.default_rng(seed)
    by, bx = (ny + block - 1) // block, (nx + block - 1) // block
    out = []
    for lo, hi in ((0.5, 1.5), (-0.2, 0.2), (-0.2, 0.2), (0.6, 1.2)):
        g = rng.uniform(lo, hi, size=(by, bx))
        out.append(np.repeat(np.repeat(g, block, axis=0), block, axis=1)[:ny, :nx].copy())
    return tuple(out)
