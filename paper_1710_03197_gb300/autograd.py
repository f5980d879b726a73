"""Differentiable forward NUFFT: y = A(om) x as a torch.autograd.Function.

Backward (both by the library's kernels):
* image gradient: A^H g (nufft_adjoint), since y is linear in x;
* trajectory gradient: Re(conj(g) dy/dom) (nufft_trajectory_gradient_grid),
  through the min-max coefficients' derivative with the neighbourhood held
  fixed.  When om needs a gradient the forward runs as its two stages
  (nufft_scale_pad_fft, nufft_interp) and keeps the oversampled spectrum F S x
  for the backward pass, which then needs no FFT of its own.
A plan is built for the given trajectory on every forward call (the
interpolator depends on om); pass ``plan`` to reuse one for a fixed om, or
``plan`` with ``refresh=True`` to move that plan to the given om first
(nufft_plan_set_trajectory: only the per-point interpolator is redone), the
form for an optimisation loop over the trajectory.
"""
from __future__ import annotations

import torch

from .plan import NufftPlan


class NufftFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, om, x, Nd, Kd, Jd, plan=None, refresh=False):
        om_c = om.detach().to(torch.float32).contiguous()
        x_c = x.detach().to(torch.complex64).contiguous()
        p = plan if plan is not None else NufftPlan(om_c, Nd, Kd, Jd)
        if plan is not None and refresh:
            p.set_trajectory(om_c)
        if ctx.needs_input_grad[0]:
            grid = p.scale_pad_fft(x_c)
            y = p.interp(grid)
            ctx.save_for_backward(grid)
        else:
            y = p.forward(x_c)
        ctx.plan = p
        return y

    @staticmethod
    def backward(ctx, gy):
        p = ctx.plan
        gy = gy.to(torch.complex64).contiguous()
        gx = p.adjoint(gy) if ctx.needs_input_grad[1] else None
        gom = None
        if ctx.needs_input_grad[0]:
            (grid,) = ctx.saved_tensors
            gom = p.trajectory_gradient_grid(grid, gy)
        return gom, gx, None, None, None, None, None


def nufft_apply(om, x, Nd, Kd, Jd, plan=None, refresh=False):
    """y = A(om) x, differentiable in om (float32, (M, d)) and x (complex64).
    refresh=True moves ``plan`` to om before applying it."""
    return NufftFunction.apply(om, x, tuple(Nd), tuple(Kd), tuple(Jd), plan, refresh)
