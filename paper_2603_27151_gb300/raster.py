"""torch.autograd.Function over the C ABI.

``DiffSoupRaster.apply(verts, tex, rast, cams, seeds, S, mode, bg)`` renders
the views with stochastic opacity masking (Eq. 5) and returns, per view, the
decoded colour features [S, C-1, H, W], a zero tensor ``logp`` [S, H, W] and
the G-buffer [S, H, W, 4].  The colour carries the first term of Eq. 8 (colour,
interior and edge gradients); ``logp`` carries the score term: a loss that adds
``(l.detach() * logp).sum()`` (value 0) hands the per-sample loss ``l`` to
Algorithm A1 2(b) as its weight.  The backward runs entirely in the library
(``ds_raster_backward`` with the forward's binning plan reused).
"""
from __future__ import annotations

import torch

from . import native as N


class Rasterizer:
    """A library context and one soup registered by reference: ``verts``
    [T, 3, 3] and ``tex`` [T, V, C] float32 CUDA tensors whose storage the
    library reads at every call (an optimiser may update them in place)."""

    def __init__(self, verts: torch.Tensor, tex: torch.Tensor, grid_n: int):
        assert verts.is_cuda and tex.is_cuda and verts.dtype == torch.float32 and tex.dtype == torch.float32
        assert verts.is_contiguous() and tex.is_contiguous()
        self.verts, self.tex, self.grid_n = verts, tex, grid_n
        self.ctx = N.Context(verts.device.index if verts.device.index is not None else torch.cuda.current_device())
        self.sid = self.ctx.soup_upload(verts, tex, grid_n, borrow=True)

    @property
    def C(self) -> int:
        return int(self.tex.shape[2])

    def close(self):
        self.ctx.close()


class DiffSoupRaster(torch.autograd.Function):
    @staticmethod
    def forward(fctx, verts, tex, rast, cams, seeds, S, mode, bg):
        if verts.data_ptr() != rast.verts.data_ptr() or tex.data_ptr() != rast.tex.data_ptr():
            raise ValueError("verts/tex must be the tensors registered with the Rasterizer")
        g, col, _ = N.alloc_outputs(cams, S, rast.C, verts.device)
        rast.ctx.raster_forward(rast.sid, cams, seeds, S, mode, bg, g, col)
        logp = [torch.zeros((S, c.height, c.width), dtype=torch.float32, device=verts.device) for c in cams]
        fctx.rast, fctx.cams, fctx.S = rast, cams, S
        fctx.save_for_backward(*g, *col)
        fctx.mark_non_differentiable(*g)
        return (*col, *logp, *g)

    @staticmethod
    def backward(fctx, *grads):
        rast, cams, S = fctx.rast, fctx.cams, fctx.S
        n = len(cams)
        saved = fctx.saved_tensors
        g, col = list(saved[:n]), list(saved[n:2 * n])
        gcol = [(gc if gc is not None else torch.zeros_like(c)).contiguous() for gc, c in zip(grads[:n], col)]
        sw = [(gl.contiguous() if gl is not None else None) for gl in grads[n:2 * n]]
        gv = torch.empty_like(rast.verts)
        gt = torch.empty_like(rast.tex)
        rast.ctx.raster_backward(rast.sid, cams, S, g, col, gcol, sw,
                                 N.DS_G_ALL | N.DS_REUSE_FORWARD | N.DS_OVERWRITE, gv, gt)
        return gv, gt, None, None, None, None, None, None


def render(rast: Rasterizer, cams, seeds, S: int = 1, mode: int = N.DS_MODE_STOCHASTIC, bg=None):
    """(colors, logps, gbufs) lists for the views ``cams``."""
    import numpy as np
    bg = np.zeros(rast.C - 1, np.float32) if bg is None else bg
    out = DiffSoupRaster.apply(rast.verts, rast.tex, rast, list(cams), seeds, S, mode, bg)
    n = len(cams)
    return list(out[:n]), list(out[n:2 * n]), list(out[2 * n:])


def l2_stochastic_loss(colors, logps, targets, S: int):
    """Mean over mask samples of the per-pixel L2 loss, plus the zero-valued
    score surrogate sum(l/S * logp): its gradient w.r.t. logp is l/S."""
    total = 0.0
    for c, lp, t in zip(colors, logps, targets):
        ell = ((c - t.unsqueeze(0)) ** 2).sum(1)          # [S, H, W]
        total = total + ell.sum() / S + (ell.detach() / S * lp).sum()
    return total
