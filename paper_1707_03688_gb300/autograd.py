"""torch.autograd wrapper around nslct_forward / nslct_backward.

``nslct_transform(x, theta, h0)`` returns y = L_theta x for a complex field x
(Nx, Ny), or a batch (B, Nx, Ny) transformed field by field, and the 10 ABCD
parameters theta (see include/nslct.h,
nslct_plan_theta); gradients flow to x and to theta through the library's
adjoint kernels (nslct_backward). PyTorch only holds memory and streams.
"""
from __future__ import annotations

import torch

from . import nslct as N


class NsLCTFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, theta, h0, precision):
        ctx.theta_device = theta.device
        ctx.theta_dtype = theta.dtype
        # a field (Nx, Ny) or a batch (B, Nx, Ny) sharing theta
        plan = N.Plan.from_theta(theta.detach().cpu().double().numpy(), x.shape[-2], x.shape[-1],
                                 h0=None if h0 is None else h0.detach().cpu().double().numpy(), precision=precision)
        y = plan.forward(x.contiguous())
        ctx.plan = plan
        ctx.save_for_backward(y)
        return y

    @staticmethod
    def backward(ctx, grad_y):
        (y,) = ctx.saved_tensors
        plan = ctx.plan
        gx, gth, _ = plan.backward(grad_y.contiguous(), y, want_theta=ctx.needs_input_grad[1])
        ctx.plan = None
        if gth is not None:
            gth = gth.to(device=ctx.theta_device, dtype=ctx.theta_dtype)
        return gx, gth, None, None


def nslct_transform(x, theta, h0=None, precision: str = "fp32"):
    """y = L_theta x with autograd for x and theta (float64 tensor of 10)."""
    return NsLCTFunction.apply(x, theta, h0, precision)
