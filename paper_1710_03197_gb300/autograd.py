"""Differentiable forward NUFFT: y = A(om) x as a torch.autograd.Function.

Backward (both by the library's kernels):
* image gradient: A^H g (nufft_adjoint), since y is linear in x;
* trajectory gradient: Re(conj(g) dy/dom) (nufft_trajectory_gradient), through
  the min-max coefficients' derivative with the neighbourhood held fixed.
A plan is built for the given trajectory on every forward call (the
interpolator depends on om); pass ``plan`` to reuse one for a fixed om.
"""
from __future__ import annotations

import torch

from .plan import NufftPlan


class NufftFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, om, x, Nd, Kd, Jd, plan=None):
        om_c = om.detach().to(torch.float32).contiguous()
        x_c = x.detach().to(torch.complex64).contiguous()
        p = plan if plan is not None else NufftPlan(om_c, Nd, Kd, Jd)
        y = p.forward(x_c)
        ctx.plan = p
        ctx.save_for_backward(x_c)
        return y

    @staticmethod
    def backward(ctx, gy):
        (x_c,) = ctx.saved_tensors
        p = ctx.plan
        gy = gy.to(torch.complex64).contiguous()
        gx = p.adjoint(gy) if ctx.needs_input_grad[1] else None
        gom = p.trajectory_gradient(x_c, gy) if ctx.needs_input_grad[0] else None
        return gom, gx, None, None, None, None


def nufft_apply(om, x, Nd, Kd, Jd, plan=None):
    """y = A(om) x, differentiable in om (float32, (M, d)) and x (complex64)."""
    return NufftFunction.apply(om, x, tuple(Nd), tuple(Kd), tuple(Jd), plan)
