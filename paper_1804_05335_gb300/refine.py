"""Differentiable candidate refinement: a torch.autograd.Function over the
library's FP64 refinement kernels (fdas_refine_fwd / fdas_refine_bwd).

P(r, z) = |sum_{k=[r]-m}^{[r]+m} A_k conj(R_z(k - r))|^2 with gradients with
respect to r, z and the spectrum A (see include/fdas.h).
"""
from __future__ import annotations

import torch

from . import fdas_half_width, fdas_refine, fdas_refine_bwd, fdas_refine_fwd


class RefinePower(torch.autograd.Function):
    """P = RefinePower.apply(spec, r, z, m): spec complex64 [nb] (device),
    r, z float64 [n] (device), m the tap half-window."""

    @staticmethod
    def forward(ctx, spec, r, z, m: int):
        spec = spec.contiguous()
        r = r.contiguous()
        z = z.contiguous()
        n = r.numel()
        P = torch.empty(n, dtype=torch.float64, device=r.device)
        dPdr = torch.empty_like(P)
        dPdz = torch.empty_like(P)
        S = torch.empty(2 * n, dtype=torch.float64, device=r.device)
        fdas_refine_fwd(spec, spec.numel(), r, z, n, m, P, dPdr, dPdz, S)
        ctx.save_for_backward(spec, r, z, dPdr, dPdz, S)
        ctx.m = int(m)
        return P

    @staticmethod
    def backward(ctx, gP):
        spec, r, z, dPdr, dPdz, S = ctx.saved_tensors
        gP = gP.contiguous().to(torch.float64)
        g_spec = g_r = g_z = None
        if ctx.needs_input_grad[0]:
            g_spec = torch.zeros_like(spec)
            fdas_refine_bwd(spec, spec.numel(), r, z, r.numel(), ctx.m, S, gP, g_spec)
        if ctx.needs_input_grad[1]:
            g_r = gP * dPdr
        if ctx.needs_input_grad[2]:
            g_z = gP * dPdz
        return g_spec, g_r, g_z, None


def refine_power(spec, r, z, m: int):
    return RefinePower.apply(spec, r, z, m)


def refine(spec, r0, z0, zmax: int = 200, steps: int = 20, lr_r: float = 0.15, lr_z: float = 9.0,
           m: int | None = None):
    """Gradient ascent from (r0, z0) in one library call; returns (r, z, P)."""
    if m is None:
        m = fdas_half_width(int(zmax))
    r0 = r0.contiguous().to(torch.float64)
    z0 = z0.contiguous().to(torch.float64)
    r = torch.empty_like(r0)
    z = torch.empty_like(z0)
    P = torch.empty_like(r0)
    fdas_refine(spec, spec.numel(), r0, z0, r0.numel(), m, steps, lr_r, lr_z, r, z, P)
    return r, z, P
