"""torch.autograd.Function over afr_reconstruct / afr_reconstruct_backward.

The forward filters the context's current frame view with widths mapped by
theta = (alpha_s, beta_s, clamp_s, alpha_t, beta_t, clamp_t); the backward
calls the hand-written adjoint, which recomputes the per-pixel weight sums
instead of storing them. Gradients and sample densities are held fixed, as
in afr_reconstruct_backward. The output's weight channel W is treated as a
constant.
"""
from __future__ import annotations

import torch

from .api import Reconstructor


class ReconstructFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, frame_colors, rec: Reconstructor, t_now: float):
        if frame_colors is not None:
            rec.set_frame_colors(frame_colors.detach())
        out = rec.reconstruct(t_now, theta)
        ctx.rec = rec
        ctx.n_frame = None if frame_colors is None else frame_colors.shape[0]
        ctx.theta_meta = (theta.device, theta.dtype)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        want_c = ctx.needs_input_grad[1]
        want_p = ctx.needs_input_grad[0]
        gcol, gprm = ctx.rec.backward(grad_out, want_colors=want_c, want_params=want_p, n_frame=ctx.n_frame)
        if gprm is not None:
            gprm = gprm.to(*ctx.theta_meta)
        return gprm, gcol, None, None


def reconstruct(rec: Reconstructor, theta: torch.Tensor, t_now: float = 1.0, frame_colors=None):
    """Differentiable reconstruction: returns the [H, W, 4] image."""
    return ReconstructFunction.apply(theta, frame_colors, rec, t_now)
