"""The differentiable training step, captured in one CUDA graph.

Workload: a 20,000-triangle soup (N = 8, 8 channels), 100 seeded cameras at
1024x768 whose targets come from a 200,000-triangle reference soup rendered
with binary opacity (Eq. 3); every step takes four views (Sec. 4 "four views
in parallel"), renders them with stochastic opacity masking, evaluates the L2
loss, runs the backward and applies Adam to vertices (lr 1e-2) and texture
logits (lr 5e-2) with beta = (0.9, 0.999), eps = 1e-8 (supplementary
"Hyperparameters").

The graph records the library calls with device-resident cameras and seeds
(the fused ds_raster_train_l2_devcam, or the separate *_devcam calls) and no
host synchronisation (DS_NO_SYNC with bin capacity reserved beforehand);
before each replay the host writes the step's
view indices and seeds into small device tensors.  ``check()`` reads the
library's status word: a bin overflow (DS_ERR_CAPACITY) makes the next
``step()`` grow the capacity and capture again.
"""
from __future__ import annotations

import numpy as np
import torch

from . import inputs as I
from . import native as N


class TrainStep:
    def __init__(self, device: str = "cuda", T: int = 20_000, T_ref: int = 200_000, n_cams: int = 100,
                 width: int = 1024, height: int = 768, per_step: int = 4, S: int = 1,
                 lr_verts: float = 1e-2, lr_tex: float = 5e-2, fused: bool = True):
        sc, ref = I.training_setup(T=T, T_ref=T_ref, n_cams=n_cams, width=width, height=height)
        self.sc, self.S, self.per_step, self.n_cams = sc, S, per_step, n_cams
        self.fused = fused   # one fused training pass per step instead of forward, loss and backward calls
        self.dev = torch.device(device)
        self.wh = [(width, height)] * per_step
        self.verts = torch.from_numpy(sc.verts).to(self.dev).contiguous()
        self.tex = torch.from_numpy(sc.tex).to(self.dev).contiguous()
        self.verts.grad = torch.zeros_like(self.verts)
        self.tex.grad = torch.zeros_like(self.tex)
        self.ctx = N.Context(self.dev.index if self.dev.index is not None else torch.cuda.current_device())
        self.sid = self.ctx.soup_upload(self.verts, self.tex, sc.grid_n, borrow=True)
        C = sc.C
        # targets of all cameras (rendered once, not part of the step)
        rv, rt = torch.from_numpy(ref.verts).to(self.dev), torch.from_numpy(ref.tex).to(self.dev)
        rsid = self.ctx.soup_upload(rv, rt, ref.grid_n)
        self.targets_all = torch.empty((n_cams, C - 1, height, width), dtype=torch.float32, device=self.dev)
        for k0 in range(0, n_cams, 8):
            cams = sc.cams[k0:k0 + 8]
            g, col, _ = N.alloc_outputs(cams, 1, C, self.dev)
            self.ctx.raster_forward(rsid, cams, None, 1, N.DS_MODE_THRESHOLD_HALF, sc.bg, g, col)
            for j, c in enumerate(col):
                self.targets_all[k0 + j].copy_(c[0])
        torch.cuda.synchronize()
        self.ctx.soup_free(rsid)
        del rv, rt
        # all cameras on the device; per-step selections
        self.cams_all = torch.from_numpy(N.camera_bytes(sc.cams)).to(self.dev)
        self.idx = torch.zeros(per_step, dtype=torch.int64, device=self.dev)
        self.seeds = torch.zeros(per_step, dtype=torch.int64, device=self.dev)
        self.cams_sel = self.cams_all.index_select(0, self.idx).contiguous()
        self.targets_sel = torch.empty((per_step, C - 1, height, width), dtype=torch.float32, device=self.dev)
        self.targets = [self.targets_sel[j] for j in range(per_step)]
        self.g = [torch.empty((S, height, width, 4), dtype=torch.int32, device=self.dev) for _ in range(per_step)]
        self.col = [torch.empty((S, C - 1, height, width), dtype=torch.float32, device=self.dev)
                    for _ in range(per_step)]
        self.gcol = [torch.empty_like(c) for c in self.col]
        self.sw = [torch.empty((S, height, width), dtype=torch.float32, device=self.dev) for _ in range(per_step)]
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        self.opt = torch.optim.Adam([{"params": [self.verts], "lr": lr_verts},
                                     {"params": [self.tex], "lr": lr_tex}],
                                    betas=(0.9, 0.999), eps=1e-8, capturable=True)
        self.graph = None
        self.step_no = 0
        self.h_idx = torch.zeros(per_step, dtype=torch.int64).pin_memory()
        self.h_seed = torch.zeros(per_step, dtype=torch.int64).pin_memory()
        self.h_done = None   # event after the last copy out of the pinned staging

    # ------------------------------------------------------------ one step
    def _body(self, no_sync: bool):
        """The work of one step on the current stream (captured or eager)."""
        mode = N.DS_MODE_STOCHASTIC | (N.DS_NO_SYNC if no_sync else 0)
        torch.index_select(self.cams_all, 0, self.idx, out=self.cams_sel)
        torch.index_select(self.targets_all, 0, self.idx, out=self.targets_sel)
        self.loss.zero_()
        if self.fused:
            self.ctx.train_l2_devcam(self.sid, self.wh, self.cams_sel, self.seeds, self.S, mode, self.sc.bg, self.g,
                                     self.col, self.targets, self.gcol, self.sw, 1.0 / self.S, self.loss,
                                     N.DS_G_ALL | N.DS_OVERWRITE, self.verts.grad, self.tex.grad)
        else:
            self.ctx.raster_forward_devcam(self.sid, self.wh, self.cams_sel, self.seeds, self.S, mode, self.sc.bg,
                                           self.g, self.col)
            N.loss_l2(self.col, self.targets, self.gcol, self.sw, self.loss, scale=1.0 / self.S)
            self.ctx.raster_backward_devcam(self.sid, self.wh, self.cams_sel, self.S, self.g, self.col, self.gcol,
                                            self.sw, N.DS_G_ALL | N.DS_REUSE_FORWARD | N.DS_OVERWRITE,
                                            self.verts.grad, self.tex.grad)
        self.opt.step()

    def _load_views(self, step: int):
        idx, seeds = I.step_views(step, self.n_cams, self.per_step)
        if self.h_done is not None:
            self.h_done.synchronize()   # the previous copy has left the pinned staging
        self.h_idx.copy_(torch.from_numpy(idx.astype(np.int64)))
        self.h_seed.copy_(torch.from_numpy(seeds.view(np.int64)))
        self.idx.copy_(self.h_idx, non_blocking=True)
        self.seeds.copy_(self.h_seed, non_blocking=True)
        self.h_done = torch.cuda.Event()
        self.h_done.record()

    def capture(self, warmup: int = 3, headroom: float = 1.5):
        """Run eager steps (sizing every buffer), reserve bin capacity with
        headroom, then capture one step in a CUDA graph."""
        side = torch.cuda.Stream(self.dev)
        side.wait_stream(torch.cuda.current_stream())
        max_pairs = 0
        with torch.cuda.stream(side):
            for k in range(warmup):
                self._load_views(self.step_no)
                self._body(no_sync=False)
                self.step_no += 1
                max_pairs = max(max_pairs, self.ctx.plan_stats()[0])
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.ctx.reserve(int(max_pairs * headroom) + 4096)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._body(no_sync=True)
        torch.cuda.synchronize()

    def step(self):
        """One captured training step (replay).  Returns nothing; the loss of
        the step is in ``self.loss`` (device)."""
        if self.graph is None:
            self.capture()
        self._load_views(self.step_no)
        self.graph.replay()
        self.step_no += 1

    def check(self) -> bool:
        """Synchronise and read the status word; on a bin overflow, drop the
        graph (the next step grows the capacity and captures again)."""
        torch.cuda.synchronize(self.dev)   # replays run on the caller's stream
        try:
            self.ctx.status()
            return True
        except N.DsError as e:
            if e.code != -4:
                raise
            self.graph = None
            return False
