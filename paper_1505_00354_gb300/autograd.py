"""Differentiable DLT / IDLT (torch.autograd) on the library's transposed kernels.

The DLT f = P c (Eq. 1, P_{kn} = P_n(x_k)) is linear, so its vector-Jacobian
product is P^T g, which the library computes with the transposed fast chain of
Sec. 4 (gbdlt_dlt_t).  The IDLT c = D_s P^T D_w f (Eq. 2 in the matrix form of
Sec. 4) has the vector-Jacobian product D_w P D_s g (gbdlt_idlt_t).  No step of
either backward runs outside the CUDA library.
"""
from __future__ import annotations

import torch

from ._binding import get_plan, _prec_of


class DLTFunction(torch.autograd.Function):
    """f = DLT(c) along the last dimension; backward: grad_c = P^T grad_f."""

    @staticmethod
    def forward(ctx, c: torch.Tensor):
        plan = get_plan(c.shape[-1], _prec_of(c), c.device)
        ctx.plan = plan
        return plan.dlt(c)

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        return ctx.plan.dlt_t(g.contiguous())


class IDLTFunction(torch.autograd.Function):
    """c = IDLT(f) along the last dimension; backward: grad_f = D_w P D_s grad_c."""

    @staticmethod
    def forward(ctx, f: torch.Tensor):
        plan = get_plan(f.shape[-1], _prec_of(f), f.device)
        ctx.plan = plan
        return plan.idlt(f)

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        return ctx.plan.idlt_t(g.contiguous())


def dlt(c: torch.Tensor) -> torch.Tensor:
    """Differentiable DLT of a CUDA tensor [..., N] (float64 or float32)."""
    return DLTFunction.apply(c)


def idlt(f: torch.Tensor) -> torch.Tensor:
    """Differentiable IDLT of a CUDA tensor [..., N] (float64 or float32)."""
    return IDLTFunction.apply(f)
