"""Differentiable render for calibration fitting: a torch.autograd.Function over the C ABI.

The forward pass writes the coefficients into the resident model (e2e_update_model) and
renders (mixed precision); the backward pass is the hand-written adjoint kernel
(e2e_render_adjoint): the vector-Jacobian product of the frame with respect to every
order-slice's mapping coefficients and PSF-width coefficients, windows held at the forward's
origins.  Parameters travel as one FP64 vector: concat(cx, cy, sx, sy) in model order.
"""
from __future__ import annotations

from typing import Sequence, Tuple

import numpy as np
import torch

from .binding import Renderer


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float64) for p in parts])


def unpack(vec: np.ndarray, n_coef: int, n_slices: int) -> Tuple[np.ndarray, ...]:
    a = n_coef
    b = 2 * n_coef
    c = b + 3 * n_slices
    return vec[:a], vec[a:b], vec[b:c], vec[c:c + 3 * n_slices]


class RenderFunction(torch.autograd.Function):
    """frames = RenderFunction.apply(params, renderer, model_id, spec_ids)  (one frame per detector)."""

    @staticmethod
    def forward(ctx, params, renderer: Renderer, mid: int, spec_ids: Sequence[int]):
        m = renderer.models[mid]
        nc = sum(len(s.cx) for s in m.slices)
        cx, cy, sx, sy = unpack(params.detach().to("cpu", torch.float64).numpy(), nc, len(m.slices))
        renderer.update(mid, cx, cy, sx, sy)
        frames = renderer.render(mid, spec_ids, "mixed", "f32")
        ctx.renderer, ctx.mid, ctx.spec_ids = renderer, mid, list(spec_ids)
        ctx.param_device = params.device
        return tuple(frames)

    @staticmethod
    def backward(ctx, *grad_frames):
        r = ctx.renderer
        dldi = [g.contiguous() if g is not None else torch.zeros_like(f)
                for g, f in zip(grad_frames, r.empty_frames(ctx.mid))]
        g = r.adjoint(ctx.mid, ctx.spec_ids, dldi)
        return torch.cat(g).to(ctx.param_device), None, None, None


def render(params: torch.Tensor, renderer: Renderer, mid: int, spec_ids: Sequence[int]):
    """Differentiable render of all detectors (tuple of FP32 frames)."""
    return RenderFunction.apply(params, renderer, mid, spec_ids)
