"""One optimisation step of the paper's full training loop, through the
library (Sec. 3.3-3.4; supplementary "Hyperparameters"):

  1. the level soup's textures composed on the finest grid and activated
     (inside the forward), then the stochastic forward of the step's views
     (Eq. 5);
  2. neural deferred shading of the colour features to RGB (Sec. 3.3);
  3. the photometric loss lambda L1 + (1 - lambda) SSIM against RGB targets
     (Eq. 10), whose per-pixel value weights the score term (Alg. A1 2(b));
  4. the shading backward to the features and parameters, then the
     rasteriser backward to the level textures and vertices (Alg. A1, Eq. 8);
  5. VectorAdam for the vertices, Adam for the level textures and the MLP,
     learning rates annealed exponentially by 100x over ``total_steps``.
     In ``step`` the level textures' Adam update runs inside the
     rasteriser backward's gradient finish (ds_raster_backward_adam), so
     their gradient is never written to memory.

Every stage is a kernel of the library; PyTorch only holds the tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import native as N
from .shade import init_params


class PaperStep:
    def __init__(self, verts, tex_levels, T: int, r_min: int, r_max: int, C: int, cams, targets, S: int = 1,
                 per_step: int = 4, total_steps: int = 10_000, lr_verts: float = 1e-3, lr_tex: float = 5e-2,
                 lr_mlp: float = 1e-2, lam: float = 0.8, params=None, seed: int = 0):
        """verts [T, 3, 3] and tex_levels (levels r_min..r_max back to back)
        float32 CUDA tensors, updated in place; cams: the training cameras;
        targets[k]: RGB [3, H, W] of camera k."""
        assert C == 8, "deferred shading takes 7 colour features and the opacity"
        self.dev = verts.device
        self.verts, self.tex = verts, tex_levels
        self.T, self.r_min, self.r_max, self.C, self.S = T, r_min, r_max, C, S
        self.cams, self.targets = list(cams), list(targets)
        self.per_step, self.total = per_step, total_steps
        self.lr = dict(verts=lr_verts, tex=lr_tex, mlp=lr_mlp)
        self.lam = lam
        self.ctx = N.Context(self.dev.index if self.dev.index is not None else torch.cuda.current_device())
        self.sid = self.ctx.soup_upload_levels(verts, tex_levels, T, r_min, r_max, C, borrow=True)
        self.params = init_params(seed, self.dev) if params is None else params
        z = torch.zeros_like
        self.m = dict(verts=z(verts), tex=z(tex_levels), mlp=z(self.params))
        self.v = dict(verts=torch.zeros(verts.numel() // 3, device=self.dev), tex=z(tex_levels), mlp=z(self.params))
        self.g_verts, self.g_tex, self.g_params = z(verts), z(tex_levels), z(self.params)
        self.loss = torch.zeros(1, device=self.dev)
        self.step_no = 0
        self.rng = np.random.default_rng(seed)

    def gradients(self, view_ids, seeds, tex_adam=None):
        """Steps 1-4 for the given views and mask seeds: fills g_verts, g_tex,
        g_params and loss (the sum over views of the mean over samples of the
        summed per-pixel loss); returns the shaded RGB images.  tex_adam =
        (lr, step): the level textures take that Adam step in the backward
        instead, and g_tex is left as it was."""
        cams = [self.cams[k] for k in view_ids]
        S, dev = self.S, self.dev
        g, col, _ = N.alloc_outputs(cams, S, self.C, dev)
        self.ctx.raster_forward(self.sid, cams, seeds, S, N.DS_MODE_STOCHASTIC, np.zeros(self.C - 1, np.float32),
                                g, col)
        rgb = [torch.empty((S, 3, c.height, c.width), device=dev) for c in cams]
        self.ctx.shade_forward(cams, self.params, col, rgb)
        g_rgb = [torch.empty_like(r) for r in rgb]
        sw = [torch.empty((S, c.height, c.width), device=dev) for c in cams]
        self.loss.zero_()
        N.loss_l1_ssim(rgb, [self.targets[k] for k in view_ids], g_rgb, sw, self.loss, lam=self.lam, scale=1.0 / S)
        g_col = [torch.empty_like(c) for c in col]
        self.ctx.shade_backward(cams, self.params, col, g_rgb, g_col, self.g_params, overwrite=True)
        flags = N.DS_G_ALL | N.DS_REUSE_FORWARD | N.DS_OVERWRITE
        if tex_adam is None:
            self.ctx.raster_backward(self.sid, cams, S, g, col, g_col, sw, flags, self.g_verts, self.g_tex)
        else:
            self.ctx.raster_backward_adam(self.sid, cams, S, g, col, g_col, sw, flags, self.m["tex"], self.v["tex"],
                                          tex_adam[0], tex_adam[1], grad_verts=self.g_verts)
        return rgb

    def step(self):
        """One step on ``per_step`` random views; returns the loss (host float)."""
        ids = self.rng.choice(len(self.cams), size=self.per_step, replace=False)
        seeds = self.rng.integers(0, 2 ** 63, size=self.per_step, dtype=np.uint64)
        self.step_no += 1
        anneal = 100.0 ** (-(self.step_no - 1) / self.total)
        self.gradients(ids, seeds, tex_adam=(self.lr["tex"] * anneal, self.step_no))
        N.adam_step(self.verts, self.g_verts, self.m["verts"], self.v["verts"], self.lr["verts"] * anneal,
                    self.step_no, dim=3)
        N.adam_step(self.params, self.g_params, self.m["mlp"], self.v["mlp"], self.lr["mlp"] * anneal, self.step_no)
        return float(self.loss)

    def close(self):
        self.ctx.close()
