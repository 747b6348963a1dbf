"""Differentiable Kelvin-Helmholtz runs: a torch.autograd.Function over the
library's adjoint (klb_adjoint_*), and the KHI initial-state recipe written
with torch operations so that autograd carries the gradient from the initial
fields to the transition-layer widths D_v, D_rho and the perturbation u_y0.

    fields = khi_fields_torch(pb, Dv, Drho, uy0)      # differentiable set-up
    ke, gamma = KLBLoss.apply(*fields, adj)           # forward: CUDA step x N
    (w_ke * ke + w_g * gamma).backward()              # reverse sweep in CUDA

Every step of the time integration and of its reverse sweep runs in the
library's kernels; torch only composes the set-up and holds device memory.
"""
from __future__ import annotations

import numpy as np
import torch

from . import inputs, klb


def khi_fields_torch(pb: inputs.Problem, Dv, Drho, uy0, device=None):
    """(rho, u_x, u_y, T) of the KHI initial state (the recipe of
    inputs.fields) as float64 tensors [ny][nx]: u_x = (u0/2) tanh(y/(D_v dy)),
    rho = (rho1+rho2)/2 + (rho1-rho2)/2 tanh(y/(D_rho dy)), T = p/rho,
    u_y = uy0 (a tensor [ny][nx])."""
    X, Y = inputs.coords(pb)
    y = torch.as_tensor(Y, dtype=torch.float64, device=device)
    Dv = torch.as_tensor(Dv, dtype=torch.float64, device=device)
    Drho = torch.as_tensor(Drho, dtype=torch.float64, device=device)
    ux = 0.5 * pb.u0 * torch.tanh(y / (Dv * pb.dy))
    rho = 0.5 * (pb.rho1 + pb.rho2) + 0.5 * (pb.rho1 - pb.rho2) * torch.tanh(y / (Drho * pb.dy))
    T = pb.p0 / rho
    uy = torch.as_tensor(uy0, dtype=torch.float64, device=device) + 0.0 * ux
    return rho, ux, uy, T


class KLBLoss(torch.autograd.Function):
    """(KE, gamma) of a run from the initial fields, with their gradients with
    respect to the four fields by the library's adjoint.  `adj` is a
    klb.KlbAdjoint sized for the run."""

    @staticmethod
    def forward(ctx, rho, ux, uy, T, adj):
        fl = [t.detach().contiguous() for t in (rho, ux, uy, T)]
        ke, gamma = adj.forward(*fl)
        adj._stamp = getattr(adj, "_stamp", 0) + 1
        adj._fresh = True
        ctx.adj, ctx.stamp = adj, adj._stamp
        ctx.save_for_backward(*fl)
        dev = rho.device
        return (torch.tensor(ke, dtype=torch.float64, device=dev),
                torch.tensor(gamma, dtype=torch.float64, device=dev))

    @staticmethod
    def backward(ctx, g_ke, g_gamma):
        adj = ctx.adj
        fl = ctx.saved_tensors
        if adj._stamp != ctx.stamp or not getattr(adj, "_fresh", True):
            adj.forward(*fl)  # the reverse sweep needs this run's checkpoints
        out = tuple(torch.empty_like(fl[0]) for _ in range(4))
        adj.backward(float(g_ke), float(g_gamma), out=out)
        adj._fresh = False
        return out[0], out[1], out[2], out[3], None


def khi_loss(pb: inputs.Problem, Dv, Drho, uy0, adj, device=None):
    """(KE, gamma) of the KHI run `pb` as a differentiable function of D_v,
    D_rho and the initial u_y field."""
    return KLBLoss.apply(*khi_fields_torch(pb, Dv, Drho, uy0, device=device), adj)
