"""torch.autograd.Function over the compositing render and its hand-written adjoint.

Forward: shw_render (COMPOSITE) with transmittance checkpoints.  Backward:
shw_render_backward, which recomputes each checkpointed segment and reverses it,
accumulating gradients for the cube, the colour map and the opacity scale.
"""
from __future__ import annotations

import torch

from . import api


class CompositeRender(torch.autograd.Function):
    @staticmethod
    def forward(ctx, cube, lut, scale, cam, kw):
        s = float(scale.detach().item()) if torch.is_tensor(scale) else float(scale)
        out = api.render(cube.detach(), cam, "composite", lut=lut.detach(), opacity_scale=s, ckpt=True,
                         scalar=False, index=False, nsamples=False, **kw)
        ctx.save_for_backward(cube, lut, out["ckpt"])
        ctx.cam, ctx.kw, ctx.s = cam, kw, s
        ctx.scale_is_tensor = torch.is_tensor(scale)
        return out["rgba"]

    @staticmethod
    def backward(ctx, grad_rgba):
        cube, lut, ckpt = ctx.saved_tensors
        g_vol = torch.zeros_like(cube) if ctx.needs_input_grad[0] else None
        g_lut = torch.zeros_like(lut) if ctx.needs_input_grad[1] else None
        g_s = torch.zeros(1, dtype=torch.float32, device=cube.device) if ctx.needs_input_grad[2] else None
        api.render_backward(cube.detach(), ctx.cam, grad_rgba.contiguous(), ckpt, lut=lut.detach(),
                            opacity_scale=ctx.s, grad_vol=g_vol, grad_lut=g_lut, grad_scale=g_s, **ctx.kw)
        if g_s is not None and ctx.scale_is_tensor:
            g_s = g_s.reshape(()).to(dtype=torch.float32)
        return g_vol, g_lut, g_s, None, None


def composite_render(cube: torch.Tensor, lut: torch.Tensor, scale, cam, **kw) -> torch.Tensor:
    """Differentiable front-to-back compositing render: returns premultiplied RGBA [H, W, 4].

    Differentiable in ``cube`` (float32 [nz, ny, nx]), ``lut`` (float32 [256, 4]) and ``scale``
    (the opacity scale, a 0-dim tensor or a float).  Keyword arguments are those of ``api.render``
    (interp, step, lo, hi, term_alpha, ckpt_interval)."""
    return CompositeRender.apply(cube, lut, scale, cam, kw)
