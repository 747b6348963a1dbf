"""Helpers shared by the GPU parity tests: run the CUDA path (through the C ABI)
and the oracle from the same seeded input, and compare them."""
from __future__ import annotations

import numpy as np

from oracle import core
from paper_1010_4124_gb300 import inputs, klb


def oracle_params(pb: inputs.Problem, eps: float = 1e-6, scheme: str = "weno5") -> core.Params:
    return core.Params(nx=pb.nx, ny=pb.ny, dx=pb.dx, dy=pb.dy, dt=pb.dt, tau=pb.tau, v=pb.v,
                       bc_x=pb.bc_x, bc_y=pb.bc_y, eps=eps, scheme=scheme)


def gpu_handle(pb: inputs.Problem, precision: str, **kw) -> klb.Klb:
    return klb.Klb.from_problem(pb, precision=precision, **kw)


def rel_err_fields(a_f, b_f, p: core.Params):
    """Relative max-norm errors ||a - b||_inf / ||b||_inf of rho, u (the velocity
    vector, |u| = sqrt(u_x^2 + u_y^2)) and T, with the fields of both states
    taken by the oracle's moments; the components u_x, u_y are reported too,
    each relative to max |u|."""
    ra, uxa, uya, Ta = core.fields(p, a_f)
    rb, uxb, uyb, Tb = core.fields(p, b_f)
    umax = np.sqrt(uxb**2 + uyb**2).max()
    umax = umax if umax > 0 else 1.0
    return {
        "rho": float(np.abs(ra - rb).max() / np.abs(rb).max()),
        "u": float(np.sqrt((uxa - uxb) ** 2 + (uya - uyb) ** 2).max() / umax),
        "T": float(np.abs(Ta - Tb).max() / np.abs(Tb).max()),
        "ux": float(np.abs(uxa - uxb).max() / umax),
        "uy": float(np.abs(uya - uyb).max() / umax),
    }


def rel_err_global(a_f, b_f):
    """||a - b||_inf over all planes / ||b||_inf over all planes (the scale of f):
    the FP32 measure, since planes whose F_k(T) is near a root carry values far
    below the others and an FP32 rounding of a large term lands on them."""
    return float(np.abs(a_f - b_f).max() / np.abs(b_f).max())


def rel_err_planes(a_f, b_f):
    """max over the 19 planes of ||a_q - b_q||_inf / ||b_q||_inf."""
    worst = 0.0
    for q in range(19):
        s = np.abs(b_f[q]).max()
        worst = max(worst, float(np.abs(a_f[q] - b_f[q]).max() / (s if s > 0 else 1.0)))
    return worst


def perturbed_state(pb: inputs.Problem, fields, seed: int, amp: float = 0.01):
    """f^(0) of the fields times (1 + amp * noise): a non-equilibrium start."""
    p = oracle_params(pb)
    f = core.init_feq(p, *fields)
    rng = np.random.default_rng(seed)
    return f * (1.0 + amp * rng.standard_normal(f.shape))
