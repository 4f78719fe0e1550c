"""Neural deferred shading (Sec. 3.3 "Neural deferred shading") as a
``torch.autograd.Function`` over ``ds_shade_forward`` / ``ds_shade_backward``.

``shade(ctx, cams, params, feats)`` maps the rasterised colour features
(per view [S, 7, H, W], e.g. the colours of ``raster.render`` with C = 8) to
RGB [S, 3, H, W] with the shared 16 -> 16 -> 16 -> 3 MLP on the features and
the SH encoding of the view direction, blended with the features' RGBA.
Gradients flow to the features (and from there into the rasteriser's
backward) and to the 595 MLP parameters.
"""
from __future__ import annotations

import math

import torch

from . import native as N

N_PARAMS = N.DS_SHADE_N_PARAMS


def init_params(seed: int = 0, device="cuda") -> torch.Tensor:
    """Xavier-uniform weights and zero biases in the parameter layout
    W1 [16][16], b1 [16], W2 [16][16], b2 [16], W3 [3][16], b3 [3]."""
    g = torch.Generator().manual_seed(seed)
    parts = []
    for o, i in ((16, 16), (16, 16), (3, 16)):
        lim = math.sqrt(6.0 / (i + o))
        parts += [(torch.rand((o, i), generator=g, dtype=torch.float64) * 2 - 1).mul_(lim).reshape(-1),
                  torch.zeros(o, dtype=torch.float64)]
    return torch.cat(parts).to(torch.float32).to(device).contiguous()


class DeferredShade(torch.autograd.Function):
    @staticmethod
    def forward(fctx, params, ctx, cams, *feats):
        feats = [f.contiguous() for f in feats]
        rgbs = [torch.empty((f.shape[0], 3, f.shape[2], f.shape[3]), dtype=torch.float32, device=f.device)
                for f in feats]
        ctx.shade_forward(cams, params, feats, rgbs)
        fctx.ctx, fctx.cams = ctx, cams
        fctx.save_for_backward(params, *feats)
        return tuple(rgbs)

    @staticmethod
    def backward(fctx, *grads):
        params, *feats = fctx.saved_tensors
        grgb = [(g if g is not None else torch.zeros((f.shape[0], 3, f.shape[2], f.shape[3]), device=f.device))
                .contiguous() for g, f in zip(grads, feats)]
        gfeat = [torch.empty_like(f) for f in feats] if any(fctx.needs_input_grad[3:]) else None
        gparams = torch.empty_like(params) if fctx.needs_input_grad[0] else None
        fctx.ctx.shade_backward(fctx.cams, params, feats, grgb, gfeat, gparams, overwrite=True)
        return (gparams, None, None, *(gfeat if gfeat is not None else [None] * len(feats)))


def shade(ctx: "N.Context", cams, params: torch.Tensor, feats):
    """RGB [S, 3, H, W] per view of the feature images ``feats``."""
    return list(DeferredShade.apply(params, ctx, list(cams), *feats))
