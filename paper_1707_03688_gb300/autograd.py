"""torch.autograd wrapper around nslct_forward / nslct_backward.

``nslct_transform(x, theta, h0)`` returns y = L_theta x for a complex field x
(Nx, Ny), or a batch (B, Nx, Ny) transformed field by field, and the 10 ABCD
parameters theta (see include/nslct.h,
nslct_plan_theta); gradients flow to x and to theta through the library's
adjoint kernels (nslct_backward). PyTorch only holds memory and streams.

With an anchor h0 for the H(theta) rule, one plan per (device, shape,
precision, h0) is kept and moved to each call's theta with
nslct_plan_theta_set (an FP64 host derivation: no allocation, no device work),
instead of a new plan per call. Without h0 every call plans afresh (H by the
Eq. HA24 search).
"""
from __future__ import annotations

import threading

import torch

from . import nslct as N

_PLANS: dict = {}
_LOCK = threading.Lock()


def _plan(theta, nx, ny, h0, precision):
    """The cached plan for this key, moved to theta (call with _LOCK held)."""
    key = (torch.cuda.current_device(), nx, ny, precision, h0.tobytes())
    plan = _PLANS.get(key)
    if plan is None:
        plan = N.Plan.from_theta(theta, nx, ny, h0=h0, precision=precision)
        _PLANS[key] = plan
    else:
        plan.set_theta(theta)
    return plan


class NsLCTFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, theta, h0, precision):
        ctx.theta_device = theta.device
        ctx.theta_dtype = theta.dtype
        th = theta.detach().cpu().double().numpy()
        nx, ny = x.shape[-2], x.shape[-1]
        # a field (Nx, Ny) or a batch (B, Nx, Ny) sharing theta
        if h0 is None:
            plan = N.Plan.from_theta(th, nx, ny, h0=None, precision=precision)
            y = plan.forward(x.contiguous())
            ctx.plan, ctx.theta = plan, None
        else:
            h0n = h0.detach().cpu().double().numpy().reshape(4)
            with _LOCK:
                plan = _plan(th, nx, ny, h0n, precision)
                y = plan.forward(x.contiguous())
            ctx.plan, ctx.theta = plan, th
        ctx.save_for_backward(y)
        return y

    @staticmethod
    def backward(ctx, grad_y):
        (y,) = ctx.saved_tensors
        plan = ctx.plan
        if ctx.theta is None:
            gx, gth, _ = plan.backward(grad_y.contiguous(), y, want_theta=ctx.needs_input_grad[1])
        else:
            # the shared plan may have moved to another call's theta since
            with _LOCK:
                plan.set_theta(ctx.theta)
                gx, gth, _ = plan.backward(grad_y.contiguous(), y, want_theta=ctx.needs_input_grad[1])
        ctx.plan = None
        if gth is not None:
            gth = gth.to(device=ctx.theta_device, dtype=ctx.theta_dtype)
        return gx, gth, None, None


def nslct_transform(x, theta, h0=None, precision: str = "fp32"):
    """y = L_theta x with autograd for x and theta (float64 tensor of 10)."""
    return NsLCTFunction.apply(x, theta, h0, precision)
