#!/usr/bin/env python
"""Benchmark of the masked rasteriser's forward + backward pass.

One step = the whole hot path on one batch: texture activation, triangle
set-up, radix-sorted tile binning, the stochastically masked raster forward
with texture decode, the fused L2 loss with its upstream gradients, and the
backward (colour, opacity-score, interior and edge gradients).  Workload: the
1080p large batch -- 100,000 triangles, 8x8 texel grids (N = 8, V = 45) of 8
FP32 channels, 4 views at 1920x1080 + 4 at 960x540, 4 mask samples per pixel.

Metric: fragments/s = covered (pixel-sample, triangle) pairs of the batch
(|F| of Eq. 1 times S) divided by the device time of a step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs the same workload with its own mask
seeds (weak scaling, no collective on the data path); rank 0 prints one JSON
line.  --impl reference times the CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

from paper_2603_27151_gb300 import inputs as I

METRIC = "fwd+bwd fragments/s"
UNIT = "fragments/s"
WORKLOAD = ("1080p large batch: 100,000 triangles, 8x8 texels x 8 FP32 channels (N=8, V=45), "
            "4x1920x1080 + 4x960x540 views, 4 mask samples/pixel, fwd+bwd, L2 loss")


# ---------------------------------------------------------------- helpers
def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest value of x over the ranks of the process group (the
    slowest rank's time); x itself when there is one rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank: float, steps: int, world: int, t_max_ms: float) -> float:
    """Whole-job throughput: the units every rank processed divided by the
    slowest rank's time."""
    return units_per_rank * steps * world / (t_max_ms / 1e3)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# The sources the tile kernels (forward, backward, edge) are compiled from.
TILE_KERNEL_SOURCES = ("ds_backward.cu", "ds_common.cuh", "ds_raster.cu", "ds_tile.cuh")


def _source_sha1() -> str:
    """Hash of the tile kernels' sources (file name and contents, sorted by
    name): the captured DRAM traffic is used only while it matches."""
    import hashlib
    h = hashlib.sha1()
    src = os.path.join(ROOT, "paper_2603_27151_gb300", "csrc")
    for f in sorted(os.path.join(src, n) for n in TILE_KERNEL_SOURCES):
        h.update(os.path.basename(f).encode())
        h.update(b"\0")
        with open(f, "rb") as fh:
            h.update(fh.read())
        h.update(b"\0")
    return h.hexdigest()


def _capture():
    """The committed ncu capture of the tile kernels (DRAM bytes and issue
    counters), or None when the kernels changed since (source hash differs)."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    return d if d.get("source_sha1") == _source_sha1() else None


def _traffic(kernel: str, pixel_samples: int):
    """DRAM bytes per launch of `kernel` from the committed ncu capture,
    scaled to this launch's pixel-samples; None when the kernels changed
    since the capture (source hash differs) or the kernel was not captured."""
    d = _capture()
    if d is None or kernel not in d.get("bytes", {}):
        return None
    return d["bytes"][kernel] * pixel_samples / d["pixel_samples"]


def _counters(kernel: str):
    """Issue and pipe counters of `kernel` from the same capture (the bound
    the kernel actually hits: issue slots, ALU/FMA/FP64 pipes, active lanes),
    or None as for _traffic."""
    d = _capture()
    if d is None or kernel not in d.get("counters", {}):
        return None
    return dict(d["counters"][kernel], source=d.get("profile"))


def workload_config(world: int) -> dict:
    """The bench line's config: the workload alone (the same for both arms)."""
    sc = I.large_batch()
    return {"workload": WORKLOAD, "triangles": sc.T, "views": len(sc.cams), "samples": sc.samples,
            "pixel_samples_per_step": sum(c.width * c.height for c in sc.cams) * sc.samples,
            "l2": "inputs larger than L2 (about 3 GB touched per step)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


# ---------------------------------------------------------------- the GPU step
class Workload:
    def __init__(self, rank: int, device: str, views: int = 0, fused: bool = True):
        import torch
        from paper_2603_27151_gb300 import native as N
        self.N = N
        self.fused = fused
        self.no_sync = False   # set once bin capacity is reserved (see reserve_bins)
        sc = I.large_batch()
        if views:
            sc.cams = sc.cams[:views]
        sc.seeds = I.mask_seeds(13 + 1000 * rank, len(sc.cams))
        self.sc = sc
        self.S = sc.samples
        self.dev = device
        self.ctx = N.Context(torch.cuda.current_device())
        self.verts = torch.from_numpy(sc.verts).to(device)
        self.tex = torch.from_numpy(sc.tex).to(device)
        self.sid = self.ctx.soup_upload(self.verts, self.tex, sc.grid_n, borrow=True)
        # targets: a second seeded soup rendered with binary opacity (Eq. 3)
        tsc = I.large_batch(soup_seed=12)
        tv, tt = torch.from_numpy(tsc.verts).to(device), torch.from_numpy(tsc.tex).to(device)
        tsid = self.ctx.soup_upload(tv, tt, tsc.grid_n)
        tg, tc, _ = N.alloc_outputs(sc.cams, 1, sc.C, device)
        self.ctx.raster_forward(tsid, sc.cams, None, 1, N.DS_MODE_THRESHOLD_HALF, sc.bg, tg, tc)
        self.targets = [c[0].contiguous() for c in tc]
        torch.cuda.synchronize()
        self.ctx.soup_free(tsid)
        del tg, tc, tv, tt
        self.g, self.col, _ = N.alloc_outputs(sc.cams, self.S, sc.C, device)
        self.gcol = [torch.empty_like(c) for c in self.col]
        self.sw = [torch.empty((self.S, c.height, c.width), dtype=torch.float32, device=device) for c in sc.cams]
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.gt = torch.zeros_like(self.tex)
        self.gv = torch.zeros_like(self.verts)
        self.cover = self.ctx.fragment_count(self.sid, sc.cams)        # |F| for one sample
        self.pairs, self.tiles = self.ctx.plan_stats()
        self.fragments = self.cover * self.S
        self.pixel_samples = sum(c.width * c.height for c in sc.cams) * self.S

    def step(self):
        """Forward, L2 loss and backward of the batch: one fused training
        pass (ds_raster_train_l2: at S = 4 the forward with the loss epilogue,
        then the backward and edge kernels), or the three separate calls."""
        N, sc = self.N, self.sc
        if self.fused:
            self.loss.zero_()
            mode = N.DS_MODE_STOCHASTIC | (N.DS_NO_SYNC if self.no_sync else 0)
            self.ctx.train_l2(self.sid, sc.cams, sc.seeds, self.S, mode, sc.bg, self.g, self.col,
                              self.targets, self.gcol, self.sw, 1.0 / self.S, self.loss,
                              N.DS_G_ALL | N.DS_OVERWRITE, self.gv, self.gt)
            return
        self.ctx.raster_forward(self.sid, sc.cams, sc.seeds, self.S, N.DS_MODE_STOCHASTIC, sc.bg, self.g, self.col)
        self.loss.zero_()
        N.loss_l2(self.col, self.targets, self.gcol, self.sw, self.loss, scale=1.0 / self.S)
        self.ctx.raster_backward(self.sid, sc.cams, self.S, self.g, self.col, self.gcol, self.sw,
                                 N.DS_G_ALL | N.DS_REUSE_FORWARD | N.DS_OVERWRITE, self.gv, self.gt)

    def reserve_bins(self, headroom: float = 1.5):
        """Reserve bin capacity for this workload (the current plan's pair
        count with headroom) so that fused steps run with DS_NO_SYNC: no host
        synchronisation inside a step.  An overflow would be reported by
        check(), never silently."""
        if not self.fused:
            return
        self.ctx.reserve(int(self.pairs * headroom) + 4096)
        self.no_sync = True

    def check(self):
        """Synchronise and raise if a no-sync step overflowed its bins."""
        import torch
        torch.cuda.synchronize()
        self.ctx.status()

    def algorithmic_bytes(self):
        """Minimum HBM bytes each stage must move per launch: the per-unit
        bytes of the scope table's measurement section (T triangles, V
        texels of C channels, C_o = C - 1 colour channels, P pixels, S
        samples, K bin pairs), with every triangle counted as visible and as
        a winner (upper bounds of T_vis and T_win).  Implementation traffic
        (staged set-up records, geometry records, texel re-reads) is not
        algorithmic and is not counted."""
        sc, S = self.sc, self.S
        T, V, C = sc.tex.shape
        Co = C - 1
        P = sum(c.width * c.height for c in sc.cams)
        nv = len(sc.cams)
        K = self.pairs
        loss = (P * 4 * Co + P * S * (4 * Co + 4)) if self.fused else 0   # fused epilogue: target in, dL/dC and l out
        fwd_raster = T * V * 4 + T * V * Co * 4 + 2 * K * 12 + P * S * (16 + 4 * Co)
        bwd_raster = P * S * (16 + 4 * Co + 4) + 2 * (36 * T + T * V * C * 4) + T * V * 4 + 2 * K * 12
        return {
            "activate": T * V * C * 4 * 2,
            "setup": nv * T * 36,
            "raster_fwd": fwd_raster + loss,
            "train": fwd_raster + loss + bwd_raster,
            "raster_bwd": bwd_raster,
            "edge_bwd": P * S * (16 + 8 * Co) + 2 * 36 * T,
            "geom": nv * T * 36,
        }

    def step_bytes(self):
        """Algorithmic bytes of one forward + backward step, as the scope
        table's measurement section states them: forward 36 T + T V 4 +
        T V C_o 4 + 2 K 12 + P S (16 + 4 C_o); backward P S (16 + 8 C_o + 4)
        + 2 (36 T + T V C 4) + T V 4."""
        sc, S = self.sc, self.S
        T, V, C = sc.tex.shape
        Co = C - 1
        P = sum(c.width * c.height for c in sc.cams)
        K = self.pairs
        fwd = 36 * T + T * V * 4 + T * V * Co * 4 + 2 * K * 12 + P * S * (16 + 4 * Co)
        bwd = P * S * (16 + 8 * Co + 4) + 2 * (36 * T + T * V * C * 4) + T * V * 4
        return fwd + bwd


def _plain_leg(wl, steps: int):
    """The same kernels on the plain path: one view per call (each call bins
    its own view and synchronises once to size its bins), no batching of
    views, no graph, default launch parameters.  Gradients are overwritten by
    the first view and accumulated by the others, as in the batched step."""
    import torch
    N, sc, S = wl.N, wl.sc, wl.S
    saved = wl.ctx.get_tuning()
    wl.ctx.set_tuning()

    def step():
        for v in range(len(sc.cams)):
            one = slice(v, v + 1)
            ow = N.DS_OVERWRITE if v == 0 else 0
            if wl.fused:
                wl.ctx.train_l2(wl.sid, sc.cams[one], sc.seeds[one], S, N.DS_MODE_STOCHASTIC, sc.bg, wl.g[one],
                                wl.col[one], wl.targets[one], wl.gcol[one], wl.sw[one], 1.0 / S, wl.loss,
                                N.DS_G_ALL | ow, wl.gv, wl.gt)
                continue
            wl.ctx.raster_forward(wl.sid, sc.cams[one], sc.seeds[one], S, N.DS_MODE_STOCHASTIC, sc.bg, wl.g[one],
                                  wl.col[one])
            N.loss_l2(wl.col[one], wl.targets[one], wl.gcol[one], wl.sw[one], wl.loss, scale=1.0 / S)
            wl.ctx.raster_backward(wl.sid, sc.cams[one], S, wl.g[one], wl.col[one], wl.gcol[one], wl.sw[one],
                                   N.DS_G_ALL | N.DS_REUSE_FORWARD | ow, wl.gv, wl.gt)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    wl.ctx.set_tuning(**saved)
    return {"value": wl.fragments / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "what": "same kernels, one view per call (%d %s per step), no graph, default launch parameters"
                    % (len(sc.cams), "fused training passes" if wl.fused else "calls of forward + loss + backward")}


# FP32 CUDA-core peak of a GB300: 152 SMs x 128 FP32 lanes x 2 flops per FMA
# at the maximum SM clock of 2070 MHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# Algorithmic flops per pixel-sample of the deferred shading MLP
# (16x16 + 16x16 + 3x16 = 560 multiply-adds): the forward; the backward =
# forward recomputation + backpropagation through W3, W2 and the feature
# columns of W1 ((48 + 256 + 112) multiply-adds) + the weight gradients (560).
SHADE_FWD_FLOPS = 2 * 560
SHADE_BWD_FLOPS = 2 * 560 + 2 * (48 + 256 + 112) + 2 * 560
# Algorithmic bytes per pixel-sample of the shading forward: 7 feature floats
# read, 3 colour floats written.
SHADE_FWD_BYTES = 4 * (7 + 3)
# Nominal dense TF32 tensor rate of a GB300 (half the bf16 rate).
TF32_NOMINAL_TFLOPS = 1125.0


def _shade_leg(wl, steps: int):
    """Neural deferred shading of the batch's colour features (S x 7 channels
    per pixel of the 8 views): forward and backward passes timed with CUDA
    events, each over ``steps`` launches (features and gradients, about
    2.5 GB, are larger than L2)."""
    import torch
    from paper_2603_27151_gb300.shade import init_params
    cams, S = wl.sc.cams, wl.S
    params = init_params(1, wl.verts.device)
    rgb = [torch.empty((S, 3, c.height, c.width), device=wl.verts.device) for c in cams]
    grgb = [torch.randn_like(r) for r in rgb]
    gfeat = [torch.empty_like(c) for c in wl.col]
    gp = torch.empty_like(params)
    N = wl.N
    path0 = wl.ctx.get_shade_path()

    def fwd_path(path):
        def f():
            wl.ctx.set_shade_path(path)
            wl.ctx.shade_forward(cams, params, wl.col, rgb)
        return f
    bwd = lambda: wl.ctx.shade_backward(cams, params, wl.col, grgb, gfeat, gp, overwrite=True)
    out = {}
    for name, fn, flops in (("forward", fwd_path(N.DS_SHADE_TENSOR_CORES), SHADE_FWD_FLOPS),
                            ("forward_cuda_cores", fwd_path(N.DS_SHADE_CUDA_CORES), SHADE_FWD_FLOPS),
                            ("backward", bwd, SHADE_BWD_FLOPS)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        tflops = flops * wl.pixel_samples / (ms / 1e3) / 1e12
        out[name] = {"ms": ms, "pixel_samples_per_s": wl.pixel_samples / (ms / 1e3),
                     "roofline": {"bound": "alu", "achieved": tflops, "peak": FP32_PEAK_TFLOPS,
                                  "unit": "TFLOP/s", "frac": tflops / FP32_PEAK_TFLOPS,
                                  "peak_kind": "nominal FP32 FMA rate at 2070 MHz",
                                  "algorithmic_flops_per_pixel_sample": flops}}
    wl.ctx.set_shade_path(path0)
    wl.ctx.status()
    # The tensor-core forward: at 28 flops per byte the MLP sits below the
    # TF32 ridge point (about 160 flops per byte), so its roofline is the
    # HBM one: 40 bytes per pixel-sample against the measured copy rate.
    hbm_peak, hbm_kind = _peaks()
    tc = out["forward"]
    gbs = SHADE_FWD_BYTES * wl.pixel_samples / (tc["ms"] / 1e3) / 1e9
    tc["roofline_flops"] = tc["roofline"]
    tc["roofline_flops"].update(peak=TF32_NOMINAL_TFLOPS, frac=tc["roofline"]["achieved"] / TF32_NOMINAL_TFLOPS,
                                bound="tensor", peak_kind="nominal dense TF32 rate")
    tc["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                      "peak_kind": hbm_kind, "algorithmic_bytes_per_pixel_sample": SHADE_FWD_BYTES}
    tc["mma"] = {"what": "per layer and tile of 128: 6 TF32 MMAs of 128 x 16 x 8 (3 products x 2 K-chunks) + 1 "
                         "for the bias; layer inputs in tensor memory", "mma_per_pixel_sample": 3 * 7 / 128}
    out["pixel_samples"] = wl.pixel_samples
    out["what"] = ("16-16-16-3 MLP on 7 features + SH2 of the view direction, RGBA blend; forward on the tensor "
                   "cores (tcgen05 kind::tf32, hi/lo split; the default path) and on the CUDA cores (FP32 FMA), "
                   "backward on the CUDA cores")
    return out


def _adapt_leg(wl):
    """One round of adaptive control (Sec. 3.4) on the batch's soup: coverage
    counts from the step's G-buffers (8 views, S = 4), view-space edge ratios
    over 20 views (the 8 views + 12 more at 1920x1080), the split/prune plan
    on the host and the rebuild
    of vertices and textures.  Device stages timed with CUDA events; the plan
    and the rebuild (which copies the plan and synchronises) with the host
    clock.  The threshold is 1/100 of the image height rather than the
    paper's 1/5, under which no edge of these 100,000 small triangles (about
    11 pixels at 1080p) would split; the budget is the current count, so the
    splits are paid for by prunes (a constant triangle count)."""
    import numpy as np
    import torch
    from paper_2603_27151_gb300 import inputs as I
    N, sc = wl.N, wl.sc
    threshold = 0.01
    T, V, C = sc.tex.shape
    cams = list(sc.cams) + [I.look_at(e, 1920, 1080) for e in I.sphere_eyes(12, 3.0, np.random.default_rng(16))]
    counts = torch.zeros(T, dtype=torch.int32, device=wl.verts.device)
    ratios = torch.empty((T, 3), device=wl.verts.device)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(2):       # warm
        counts.zero_()
        N.coverage_count(wl.g, T, counts)
        N.edge_ratios(wl.verts, cams, ratios)
    counts.zero_()
    torch.cuda.synchronize()
    ev[0].record()
    N.coverage_count(wl.g, T, counts)
    ev[1].record()
    N.edge_ratios(wl.verts, cams, ratios)
    ev[2].record()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = N.adapt_plan(counts.cpu().numpy(), ratios.cpu().numpy(), threshold, T)
    t1 = time.perf_counter()
    n = len(plan)
    vo = torch.empty((n, 3, 3), device=wl.verts.device)
    to = torch.empty((n, V, C), device=wl.verts.device)
    wl.ctx.soup_rebuild(wl.verts, wl.tex, T, [sc.grid_n], C, plan, vo, to)
    t2 = time.perf_counter()
    wl.ctx.soup_rebuild(wl.verts, wl.tex, T, [sc.grid_n], C, plan, vo, to)
    t3 = time.perf_counter()
    cov_ms = ev[0].elapsed_time(ev[1])
    peak, peak_kind = _peaks()
    cov_bytes = 16 * wl.pixel_samples + 4 * T        # G-buffer texels read (ids interleaved), counts written
    return {"coverage_ms": cov_ms, "edge_ratios_ms": ev[1].elapsed_time(ev[2]), "plan_ms": (t1 - t0) * 1e3,
            "rebuild_ms": (t3 - t2) * 1e3, "first_rebuild_ms": (t2 - t1) * 1e3,
            "triangles_in": T, "triangles_out": n, "splits": int(((plan & 7) == 1).sum() + ((plan & 7) == 3).sum()
                                                               + ((plan & 7) == 5).sum()),
            "views_measured": len(cams), "threshold": threshold,
            "coverage_roofline": {"bound": "hbm", "achieved": cov_bytes / (cov_ms / 1e3) / 1e9, "peak": peak,
                                  "unit": "GB/s", "frac": cov_bytes / (cov_ms / 1e3) / 1e9 / peak,
                                  "peak_kind": peak_kind},
            "what": "coverage over the step's G-buffers, edge ratios over 20 views, host plan (budget = current "
                    "count), rebuild"}


def _loss_optim_leg(wl, reps: int = 10):
    """The paper's loss and optimisers on the batch: lambda L1 + (1 - lambda)
    SSIM (Eq. 10) with its gradients over the step's colours (8 views, S = 4,
    7 channels), and one Adam step of the texture logits plus one VectorAdam
    step of the vertices (with the step's gradients).  CUDA events, mean over
    ``reps`` launches."""
    import torch
    N = wl.N
    T, V, C = wl.sc.tex.shape
    gcol = [torch.empty_like(c) for c in wl.col]
    sw = [torch.empty((wl.S, c.height, c.width), device=wl.verts.device) for c in wl.sc.cams]
    loss = torch.zeros(1, device=wl.verts.device)
    tex, verts = wl.tex.clone(), wl.verts.clone()
    mt, vt = torch.zeros_like(tex), torch.zeros_like(tex)
    mv, vv = torch.zeros_like(verts), torch.zeros(T * 3, device=wl.verts.device)

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ssim_ms = timed(lambda: N.loss_l1_ssim(wl.col, wl.targets, gcol, sw, loss, scale=1.0 / wl.S))
    step = [0]

    def adam():
        step[0] += 1
        N.adam_step(tex, wl.gt, mt, vt, 0.05, step[0], dim=1)
        N.adam_step(verts, wl.gv, mv, vv, 1e-3, step[0], dim=3)
    adam_ms = timed(adam)
    peak, peak_kind = _peaks()
    n_tex, n_vec = T * V * C, T * 3
    adam_bytes = 28 * n_tex + 68 * n_vec
    px = wl.pixel_samples
    return {"l1_ssim_ms": ssim_ms, "l1_ssim_pixel_samples_per_s": px / (ssim_ms / 1e3),
            "adam_ms": adam_ms, "adam_values": n_tex + 3 * n_vec,
            "adam_roofline": {"bound": "hbm", "achieved": adam_bytes / (adam_ms / 1e3) / 1e9, "peak": peak,
                              "unit": "GB/s", "frac": adam_bytes / (adam_ms / 1e3) / 1e9 / peak,
                              "peak_kind": peak_kind},
            "what": "fused L1+SSIM loss with gradients and score weights (11x11 Gaussian, 7 channels); Adam on "
                    "the texture logits + VectorAdam on the vertices"}


# ---------------------------------------------------------------- the small configurations
def _config_scenes(name: str):
    """(scene, target scene) of the 64-triangle plain workload ("plain
    small") or of the 2,000-triangle batched views ("batched views")."""
    if name == "plain_small":
        return I.plain_small(), I.plain_small(soup_seed=1)
    return I.batched_views(), I.batched_views(soup_seed=4)


def _oracle_view(job):
    """CPU oracle (bbox-scan mode) on one whole view of a small
    configuration: forward + L2 loss + backward with every gradient term,
    the target rendered first, untimed.  Returns (fragments, seconds)."""
    import oracle as O
    name, v = job
    sc, tsc = _config_scenes(name)
    cam, S = sc.cams[v], sc.samples
    tg = O.forward(tsc.verts, tsc.tex, tsc.grid_n, [cam], np.zeros(1, np.uint64), S=1,
                   mode=O.MODE_THRESHOLD_HALF, bg=sc.bg, scan=True)[0]["color"][0]
    t0 = time.perf_counter()
    f = O.forward(sc.verts, sc.tex, sc.grid_n, [cam], sc.seeds[v:v + 1], S=S, bg=sc.bg, scan=True)[0]
    d = f["color"] - tg[None]
    gc = (2.0 * d / S).astype(np.float32)
    sw = ((d.astype(np.float64) ** 2).sum(1) / S).astype(np.float32)
    O.backward(sc.verts, sc.tex, sc.grid_n, [cam], S, [f], [gc], [sw], scan=True)
    return int(f["n_cover"].sum()), time.perf_counter() - t0


def _config_cpu(name: str, n_views: int):
    """The oracle on the whole configuration: every view on its own process
    (all cores), and the same views one after another on one core."""
    import oracle as O
    O.build()
    jobs = [(name, v) for v in range(n_views)]
    cores = min(_cores(), n_views)
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_view, jobs[:1])                  # workers warm (library loaded)
        t0 = time.perf_counter()
        res = pool.map(_oracle_view, jobs)
        wall = time.perf_counter() - t0
    frags = sum(r[0] for r in res)
    one = [_oracle_view(j) for j in jobs]
    f1, s1 = sum(r[0] for r in one), sum(r[1] for r in one)
    return {"value": frags / wall, "unit": UNIT, "cores": cores, "seconds": wall,
            "cores_1": {"value": f1 / s1, "unit": UNIT, "cores": 1, "seconds": s1},
            "kind": "oracle (bbox-scan mode), whole configuration, forward + L2 loss + backward"}


def _config_leg(name: str, device: str, steps: int, tune: bool = True):
    """fwd+bwd fragments/s of a small configuration on the GPU (one fused
    training pass over all views per step, autotuned launch parameters),
    on the plain path (one view per call, default launch parameters) and in
    the CPU oracle.  CUDA events over ``steps`` steps after 5 warm-up
    steps; the inputs stay resident (these configurations fit in L2, so the
    numbers are L2-resident by construction)."""
    import torch
    from paper_2603_27151_gb300 import autotune
    from paper_2603_27151_gb300 import native as N
    sc, tsc = _config_scenes(name)
    S, C = sc.samples, sc.C
    ctx = N.Context(torch.cuda.current_device())
    verts, tex = torch.from_numpy(sc.verts).to(device), torch.from_numpy(sc.tex).to(device)
    sid = ctx.soup_upload(verts, tex, sc.grid_n, borrow=True)
    tv, tt = torch.from_numpy(tsc.verts).to(device), torch.from_numpy(tsc.tex).to(device)
    tsid = ctx.soup_upload(tv, tt, tsc.grid_n)
    tg, tc, _ = N.alloc_outputs(sc.cams, 1, C, device)
    ctx.raster_forward(tsid, sc.cams, None, 1, N.DS_MODE_THRESHOLD_HALF, sc.bg, tg, tc)
    targets = [c[0].contiguous() for c in tc]
    g, col, _ = N.alloc_outputs(sc.cams, S, C, device)
    gcol = [torch.empty_like(c) for c in col]
    sw = [torch.empty((S, c.height, c.width), device=device) for c in sc.cams]
    loss = torch.zeros(1, device=device)
    gt, gv = torch.zeros_like(tex), torch.zeros_like(verts)
    fragments = ctx.fragment_count(sid, sc.cams) * S

    def batched():
        loss.zero_()
        ctx.train_l2(sid, sc.cams, sc.seeds, S, N.DS_MODE_STOCHASTIC, sc.bg, g, col, targets, gcol, sw, 1.0 / S,
                     loss, N.DS_G_ALL | N.DS_OVERWRITE, gv, gt)

    def plain():
        loss.zero_()
        for v in range(len(sc.cams)):
            one = slice(v, v + 1)
            ctx.train_l2(sid, sc.cams[one], sc.seeds[one], S, N.DS_MODE_STOCHASTIC, sc.bg, g[one], col[one],
                         targets[one], gcol[one], sw[one], 1.0 / S, loss,
                         N.DS_G_ALL | (N.DS_OVERWRITE if v == 0 else 0), gv, gt)

    def timed(fn):
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    ctx.set_tuning()
    plain_ms = timed(plain)
    tuning = None
    if tune:
        batched()
        tuning = autotune.tuned(ctx, sid, sc.T, sc.grid_n, C, sc.cams, sc.seeds, S, N.DS_MODE_STOCHASTIC, sc.bg, g,
                                col, gcol, sw, gv, gt, reps=3, targets=targets, scale=1.0 / S)
    batched_ms = timed(batched)
    ctx.close()
    px = sum(c.width * c.height for c in sc.cams)
    return {"gpu": {"value": fragments / (batched_ms / 1e3), "unit": UNIT, "ms_per_step": batched_ms,
                    "tuning": tuning},
            "gpu_plain": {"value": fragments / (plain_ms / 1e3), "unit": UNIT, "ms_per_step": plain_ms},
            "batched_speedup": plain_ms / batched_ms,
            "fragments_per_step": fragments, "pixel_samples_per_step": px * S, "views": len(sc.cams),
            "triangles": sc.T}


def widened_cases():
    """One launch of each kernel of the widened rows on a case larger than L2
    (for profiler captures; prints one check line, not a bench line): deferred
    shading forward (tensor cores, then CUDA cores) and backward of two
    1920x1080 views at S = 4; the L1 +
    SSIM loss of the same images (7 channels); the level composition
    (standalone and inside the activation of a level soup, 20,000 triangles,
    levels 2..5) and its adjoint; coverage counts of the 2-view G-buffers; one
    Adam step of 36.9 M values."""
    import numpy as np
    import torch
    from paper_2603_27151_gb300 import inputs as I
    from paper_2603_27151_gb300 import native as N
    from paper_2603_27151_gb300.shade import init_params
    torch.cuda.set_device(0)
    dev = "cuda"
    cams = I.large_batch().cams[:2]
    S = 4
    ctx = N.Context(0)
    gen = torch.Generator(device=dev).manual_seed(1)
    feats = [torch.rand((S, 7, c.height, c.width), generator=gen, device=dev) for c in cams]
    rgb = [torch.empty((S, 3, c.height, c.width), device=dev) for c in cams]
    grgb = [torch.randn(r.shape, generator=gen, device=dev) for r in rgb]
    gf = [torch.empty_like(f) for f in feats]
    params = init_params(1)
    gp = torch.empty_like(params)
    ctx.shade_forward(cams, params, feats, rgb)                 # tensor cores (the default)
    ctx.set_shade_path(N.DS_SHADE_CUDA_CORES)
    ctx.shade_forward(cams, params, feats, rgb)                 # FP32 FMA
    ctx.set_shade_path(N.DS_SHADE_TENSOR_CORES)
    ctx.shade_backward(cams, params, feats, grgb, gf, gp, overwrite=True)
    tg = [torch.rand((7, c.height, c.width), generator=gen, device=dev) for c in cams]
    sw = [torch.empty((S, c.height, c.width), device=dev) for c in cams]
    loss = torch.zeros(1, device=dev)
    N.loss_l1_ssim(feats, tg, gf, sw, loss, scale=1.0 / S)
    T, C = 20000, 8
    lv = I.level_logits(T, 2, 5, C, np.random.default_rng(2))
    tex = torch.from_numpy(np.concatenate([l.reshape(-1) for l in lv])).to(dev)
    fine = torch.empty((T, N.level_V(5), C), device=dev)
    N.levels_compose(tex, T, 2, 5, C, fine, activate=True)
    verts = torch.from_numpy(I.box_soup(T, 0.05, np.random.default_rng(3))).to(dev)
    sid = ctx.soup_upload_levels(verts, tex, T, 2, 5, C, borrow=True)
    g, col, _ = N.alloc_outputs(cams, 1, C, dev)
    ctx.raster_forward(sid, cams, None, 1, N.DS_MODE_THRESHOLD_HALF, np.zeros(C - 1, np.float32), g, col)
    gcol = [torch.randn(c.shape, generator=gen, device=dev) for c in col]
    gt = torch.empty_like(tex)
    ctx.raster_backward(sid, cams, 1, g, col, gcol, None, N.DS_G_TEX | N.DS_REUSE_FORWARD | N.DS_OVERWRITE, None, gt)
    counts = torch.zeros(T, dtype=torch.int32, device=dev)
    N.coverage_count(g, T, counts)
    x = torch.randn(36_900_000, generator=gen, device=dev)
    gx = torch.randn(x.shape, generator=gen, device=dev)
    m, v = torch.zeros_like(x), torch.zeros_like(x)
    N.adam_step(x, gx, m, v, 0.05, 1)
    torch.cuda.synchronize()
    ctx.status()
    print("widened cases ok: loss %.6g, |grad params| %.6g, |grad levels| %.6g, coverage %d"
          % (float(loss), float(gp.abs().sum()), float(gt.abs().sum()), int(counts.sum())))


def _paper_step_leg(device: str, steps: int):
    """The paper's full training step through the library (paper_step.py):
    a level soup (100,000 triangles, levels 2..5), 4 views of 1920x1080 per
    step drawn from the batch's 8 cameras, S = 1, deferred shading, L1 + SSIM
    against RGB targets, both backward passes, VectorAdam + Adam.  Timed with
    CUDA events over ``steps`` steps after 2 warm-up steps."""
    import numpy as np
    import torch
    from paper_2603_27151_gb300 import inputs as I
    from paper_2603_27151_gb300.paper_step import PaperStep
    sc = I.large_batch()
    cams = [c for c in sc.cams if c.width == 1920]
    T, C, r_min, r_max = sc.T, 8, 2, 5
    lv = I.level_logits(T, r_min, r_max, C, np.random.default_rng(14))
    verts = torch.from_numpy(sc.verts).to(device)
    tex = torch.from_numpy(np.concatenate([l.reshape(-1) for l in lv])).to(device)
    del lv
    gen = torch.Generator(device=device).manual_seed(17)
    targets = [torch.rand((3, c.height, c.width), generator=gen, device=device) for c in cams]
    st = PaperStep(verts, tex, T, r_min, r_max, C, cams, targets, S=1, per_step=4, total_steps=10_000)
    losses = [st.step() for _ in range(2)]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        losses.append(st.step())
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    st.close()
    return {"ms_per_step": ms, "steps_per_s": 1e3 / ms, "views_per_step": 4, "triangles": T, "levels": [r_min, r_max],
            "loss_first": losses[0], "loss_last": losses[-1],
            "what": "forward (level composition in the activation) + deferred shading + L1/SSIM + shading and "
                    "rasteriser backward + VectorAdam/Adam; 4 x 1920x1080 views, S = 1; the step reads its loss "
                    "back to the host"}


def _levels_leg(device: str, steps: int):
    """The 1080p batch with a multi-resolution texture: levels 2..5 (the last
    stage of the coarse-to-fine schedule; finest grid 32 subdivisions, 561
    feature vertices per triangle), fused training steps.  The composition
    (activation stage) and its adjoint (finish stage) are timed by the
    library's stage profiler (CUDA events around each stage)."""
    import numpy as np
    import torch
    from paper_2603_27151_gb300 import inputs as I
    from paper_2603_27151_gb300 import native as N
    sc = I.large_batch()
    T, C, S, r_min, r_max = sc.T, 8, sc.samples, 2, 5
    lv = I.level_logits(T, r_min, r_max, C, np.random.default_rng(14))
    ctx = N.Context(torch.cuda.current_device())
    verts = torch.from_numpy(sc.verts).to(device)
    tex = torch.from_numpy(np.concatenate([l.reshape(-1) for l in lv])).to(device)
    del lv
    sid = ctx.soup_upload_levels(verts, tex, T, r_min, r_max, C, borrow=True)
    gen = torch.Generator(device=device).manual_seed(15)
    targets = [torch.rand((C - 1, c.height, c.width), generator=gen, device=device) for c in sc.cams]
    g, col, _ = N.alloc_outputs(sc.cams, S, C, device)
    gcol = [torch.empty_like(c) for c in col]
    sw = [torch.empty((S, c.height, c.width), device=device) for c in sc.cams]
    loss = torch.zeros(1, device=device)
    gt, gv = torch.empty_like(tex), torch.empty_like(verts)

    def step():
        loss.zero_()
        ctx.train_l2(sid, sc.cams, sc.seeds, S, N.DS_MODE_STOCHASTIC, sc.bg, g, col, targets, gcol, sw, 1.0 / S,
                     loss, N.DS_G_ALL | N.DS_OVERWRITE, gv, gt)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    ctx.profile_reset()
    ctx.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ctx.profile(False)
    prof = ctx.profile_read()
    ms = e0.elapsed_time(e1) / steps
    sum_v = sum(N.level_V(R) for R in range(r_min, r_max + 1))
    vf = N.level_V(r_max)
    peak, peak_kind = _peaks()
    algo = {"activate": 4 * C * T * sum_v + T * vf * (4 * C + 4),          # levels in, act + opacity plane out
            "finish": 8 * C * T * vf + 4 * C * T * sum_v + 12 * 9 * T}      # FP64 fine gradient in, levels out
    out = {"ms_per_step": ms, "levels": [r_min, r_max], "feature_vertices": vf, "triangles": T,
           "what": "fused training steps of the 1080p batch on a level soup (compose in the activation, "
                   "adjoint in the gradient finish)"}
    for stage, b in algo.items():
        runs, tot = prof.get(stage, (0, 0.0))
        if runs:
            lms = tot / runs
            out[stage] = {"ms": lms, "algorithmic_bytes": b,
                          "roofline": {"bound": "hbm", "achieved": b / (lms / 1e3) / 1e9, "peak": peak,
                                       "unit": "GB/s", "frac": b / (lms / 1e3) / 1e9 / peak, "peak_kind": peak_kind}}
    ctx.close()
    return out


def _train_leg(device: str, iters: int, fused: bool = True):
    """The captured training step (20,000 triangles, 4 views of 1024x768 per
    step drawn from 100 cameras, Adam) against the same step run eagerly."""
    import torch
    from paper_2603_27151_gb300.train import TrainStep
    ts = TrainStep(device, fused=fused)
    ts.capture(warmup=3)
    for _ in range(3):
        ts.step()
    torch.cuda.synchronize()
    l0 = float(ts.loss.item())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(iters):
        ts.step()
    e1.record()
    ok = ts.check()
    ms = e0.elapsed_time(e1) / iters
    l1 = float(ts.loss.item())
    # eager: the same body without the graph (host launches, one bin-sizing
    # synchronisation per forward)
    e0.record()
    n_eager = max(5, iters // 4)
    for _ in range(n_eager):
        ts._load_views(ts.step_no)
        ts._body(no_sync=False)
        ts.step_no += 1
    e1.record()
    torch.cuda.synchronize()
    ms_eager = e0.elapsed_time(e1) / n_eager
    px = ts.per_step * 1024 * 768
    # algorithmic bytes of one step: the fused pass (forward, loss, texture,
    # score and interior terms), the edge terms and the optimiser's update
    T, V, C = ts.tex.shape
    Co, nv = C - 1, ts.per_step
    K = ts.ctx.plan_stats()[0]
    step_bytes = (K * (8 + 64) + T * V * 4 + T * V * C * 4 * 3 + px * (16 + 4 * Co) + px * 4 * Co
                  + px * (4 * Co + 4) + 36 * T * 2 + nv * T * (36 + 208)
                  + px * (16 + 8 * Co) + nv * T * (64 + 208)
                  + (T * V * C + 9 * T) * 4 * 4)   # Adam: parameter, gradient and two moments
    peak, peak_kind = _peaks()
    return {"iters_per_s": 1e3 / ms, "ms_per_iter": ms, "pixels_per_s": px / (ms / 1e3),
            "hbm_frac": step_bytes / (ms / 1e3) / 1e9 / peak, "hbm_bytes_per_iter": step_bytes,
            "eager_iters_per_s": 1e3 / ms_eager, "eager_ms_per_iter": ms_eager, "status_ok": ok,
            "loss_before": l0, "loss_after": l1,
            "what": "20,000 triangles (N=8, C=8), 4 of 100 views at 1024x768 per step, S=1, L2 loss, Adam; "
                    "one CUDA graph per step vs the same step launched eagerly"}


def _request_fragments(device, soups, reqs):
    """Covered (pixel, triangle) pairs of each request's view (|F| of Eq. 1,
    one sample), counted by the library on a separate context, summed over
    the requests."""
    import torch
    from paper_2603_27151_gb300 import native as N
    ctx = N.Context(torch.cuda.current_device())
    total = 0
    by_soup = {}
    for (_, k, cam, _) in reqs:
        by_soup.setdefault(k, []).append(cam)
    for k, cams in by_soup.items():
        sc = soups[k]
        v, t = torch.from_numpy(sc.verts).to(device), torch.from_numpy(sc.tex).to(device)
        sid = ctx.soup_upload(v, t, sc.grid_n, borrow=True)
        for i in range(0, len(cams), 64):
            total += ctx.fragment_count(sid, cams[i:i + 64])
        ctx.soup_free(sid)
    ctx.close()
    return total


def _serve_run(device, soups, reqs, plain: bool, time_scale: float = 1.0):
    """Replay ``reqs`` through the batching server (4 worker streams, up to
    16 same-soup requests per launch, 8 GiB admission budget) or the plain
    server (one stream, one request per launch)."""
    import torch
    from paper_2603_27151_gb300 import native as N
    from paper_2603_27151_gb300.serve import SlotPool, replay
    if plain:
        srv = N.Server(torch.cuda.current_device(), n_streams=1, mem_budget=8 << 30, max_batch=1,
                       reserve_pairs=1 << 22)
    else:
        srv = N.Server(torch.cuda.current_device(), n_streams=4, mem_budget=8 << 30, max_batch=16,
                       reserve_pairs=1 << 22)
    ids = [srv.add_soup(torch.from_numpy(sc.verts).to(device), torch.from_numpy(sc.tex).to(device), sc.grid_n)
           for sc in soups]
    pool = SlotPool(I.SERVE_RESOLUTIONS, 48, 8, device)
    # warm-up: every soup at every resolution (sizes each worker's scratch)
    warm = [(0.0, k, I.look_at(np.array([0.0, -3.0, 0.5]), w, h), 1) for k in range(len(soups))
            for (w, h) in I.SERVE_RESOLUTIONS]
    replay(srv, ids, warm * 2, pool, time_scale=0.0)
    r = replay(srv, ids, reqs, pool, time_scale=time_scale)
    srv.close()
    return r


def _serve_stats(r, fragments: int, offered):
    lat = r["latency_ms"]
    n = len(lat)
    bytes_per_px = 16 + 4 * 7
    out_bytes = float(r["pixels"].sum()) * bytes_per_px
    return {"requests": n, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "frames_per_s": n / r["span_s"],
            "pixels_per_s": float(r["pixels"].sum()) / r["span_s"],
            "fragments_per_s": fragments / r["span_s"],
            "output_gbs": out_bytes / r["span_s"] / 1e9,
            "hbm_frac": out_bytes / r["span_s"] / 1e9 / _peaks()[0],
            "mean_batch": float(r["batch"].mean()), "offered_rps": offered}


def _serve_leg(device: str, seconds: float, plain: bool):
    """Replay the Poisson request stream (16 resident soups, 2000 requests/s,
    resolutions 256^2 .. 1920x1080, forward with binary opacity)."""
    soups, reqs = I.serving_workload(duration=seconds)
    r = _serve_run(device, soups, reqs, plain)
    out = _serve_stats(r, _request_fragments(device, soups, reqs), len(reqs) / seconds)
    out["what"] = ("plain: one stream, one request per launch" if plain else
                   "4 worker streams, up to 16 same-soup requests per launch, 8 GiB admission budget")
    return out


def _serve_sweep(device: str):
    """The same stream at higher Poisson rates, and closed loop (every request
    submitted at once: the server saturated), through the batching server and
    the plain server.  fragments/s counts the covered (pixel, triangle)
    pairs of the served views; hbm_frac is the output bytes (G-buffer and
    colour) per second over the measured HBM bandwidth."""
    out = []
    for rate, secs in ((8000.0, 2.5), (20000.0, 1.5), (None, 0.0)):
        if rate is None:
            soups, reqs = I.serving_workload(rate=4000.0, duration=1.0, arrival_seed=41)
            scale, offered = 0.0, "closed loop (all submitted at once)"
        else:
            soups, reqs = I.serving_workload(rate=rate, duration=secs, arrival_seed=41)
            scale, offered = 1.0, len(reqs) / secs
        frags = _request_fragments(device, soups, reqs)
        row = {"offered_rps": offered}
        for plain in (False, True):
            r = _serve_run(device, soups, reqs, plain, time_scale=scale)
            row["plain" if plain else "batching"] = _serve_stats(r, frags, offered)
        out.append(row)
    return out


def _gpu_arm(args):
    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = "cuda:%d" % local
    from paper_2603_27151_gb300 import native as N
    wl = Workload(rank, dev, args.views, fused=not args.unfused)
    tuning = None
    if args.tuning:
        tw, db, bps, ch = (int(x) for x in args.tuning.split(","))
        wl.ctx.set_tuning(tw, db, bps, ch)
        tuning = dict(wl.ctx.get_tuning(), cached=None)
    elif not args.no_tune:
        # launch parameters from the autotuner (cached per workload); untimed
        from paper_2603_27151_gb300 import autotune
        wl.step()
        tuning = autotune.tuned(wl.ctx, wl.sid, wl.sc.T, wl.sc.grid_n, wl.sc.C, wl.sc.cams, wl.sc.seeds, wl.S,
                                N.DS_MODE_STOCHASTIC, wl.sc.bg, wl.g, wl.col, wl.gcol, wl.sw, wl.gv, wl.gt, reps=2,
                                targets=wl.targets if wl.fused else None, scale=1.0 / wl.S)
    wl.step()
    wl.pairs, wl.tiles = wl.ctx.plan_stats()   # bin pairs with the chosen tiles
    wl.reserve_bins()
    for _ in range(args.warmup):
        wl.step()
    wl.check()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-timed steps (inputs resident in HBM; working set > L2)
    wl.ctx.profile_reset()
    wl.ctx.profile(True)
    launches0 = N.kernel_launches()
    stream = torch.cuda.current_stream()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]   # one pair per step
    barrier()
    with ClockSampler(local) as clk:
        evs[0].record(stream)
        for k in range(args.steps):
            wl.step()
            evs[k + 1].record(stream)
        torch.cuda.synchronize()
    launches = N.kernel_launches() - launches0
    wl.check()
    wl.ctx.profile(False)
    prof = wl.ctx.profile_read()
    ms = evs[0].elapsed_time(evs[-1])
    step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    t_max = max_over_ranks(ms, world, dev)
    barrier()

    # ---- end to end through the public API with host buffers.  Every step
    # copies its inputs (vertices, texture logits, targets) from pinned host
    # memory and its results (the texture and vertex gradients and the loss)
    # back to pinned host memory, and the host reads the loss.
    #  serial:    copy in -> step -> copy out on one stream, then the host
    #             waits: nothing overlaps;
    #  pipelined: inputs and gradients double buffered: step k+1's inputs
    #             are copied on a copy stream while step k computes, and step
    #             k's gradients are copied out on a third stream while step
    #             k+1 computes, as a training loop with a prefetching loader
    #             and an asynchronous parameter server would run.
    hv = wl.verts.cpu().pin_memory()
    ht = wl.tex.cpu().pin_memory()
    htg = [x.cpu().pin_memory() for x in wl.targets]
    h2d = hv.numel() * 4 + ht.numel() * 4 + sum(x.numel() * 4 for x in htg)
    hgt = [torch.empty(wl.gt.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    hgv = [torch.empty(wl.gv.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    hl = [torch.zeros(1, dtype=torch.float32).pin_memory() for _ in range(2)]
    d2h = wl.gt.numel() * 4 + wl.gv.numel() * 4 + 4
    comp = torch.cuda.current_stream()

    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        wl.verts.copy_(hv, non_blocking=True)
        wl.tex.copy_(ht, non_blocking=True)
        for d, h in zip(wl.targets, htg):
            d.copy_(h, non_blocking=True)
        wl.step()
        hgt[0].copy_(wl.gt, non_blocking=True)
        hgv[0].copy_(wl.gv, non_blocking=True)
        hl[0].copy_(wl.loss, non_blocking=True)
        comp.synchronize()
        _ = float(hl[0][0])
    e2e_serial_s = time.perf_counter() - t0
    wl.check()
    e2e_serial_s = max_over_ranks(e2e_serial_s, world, dev)

    home = (wl.verts, wl.tex, wl.targets, wl.sid, wl.gt, wl.gv, wl.loss)
    bufs = [home]
    v2, t2 = torch.empty_like(wl.verts), torch.empty_like(wl.tex)
    bufs.append((v2, t2, [torch.empty_like(x) for x in wl.targets],
                 wl.ctx.soup_upload(v2, t2, wl.sc.grid_n, borrow=True),
                 torch.empty_like(wl.gt), torch.empty_like(wl.gv), torch.zeros_like(wl.loss)))
    copy, back = torch.cuda.Stream(), torch.cuda.Stream()
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    freed = [torch.cuda.Event(), torch.cuda.Event()]
    stepped = [torch.cuda.Event(), torch.cuda.Event()]
    readback = [torch.cuda.Event(), torch.cuda.Event()]

    def load_inputs(b):
        v, t, tg = bufs[b][:3]
        with torch.cuda.stream(copy):
            copy.wait_event(freed[b])   # the step that last read buffer b has finished
            v.copy_(hv, non_blocking=True)
            t.copy_(ht, non_blocking=True)
            for d, h in zip(tg, htg):
                d.copy_(h, non_blocking=True)
            copied[b].record(copy)

    for b in range(2):
        freed[b].record(comp)
        readback[b].record(comp)
    barrier()
    t0 = time.perf_counter()
    load_inputs(0)
    for k in range(args.steps):
        b = k % 2
        if k + 1 < args.steps:
            load_inputs(1 - b)
        comp.wait_event(copied[b])
        comp.wait_event(readback[b])    # step k-2's gradients have left buffer b
        wl.verts, wl.tex, wl.targets, wl.sid, wl.gt, wl.gv, wl.loss = bufs[b]
        wl.step()
        freed[b].record(comp)
        stepped[b].record(comp)
        with torch.cuda.stream(back):
            back.wait_event(stepped[b])
            hgt[b].copy_(wl.gt, non_blocking=True)
            hgv[b].copy_(wl.gv, non_blocking=True)
            hl[b].copy_(wl.loss, non_blocking=True)
            readback[b].record(back)
        if k >= 1:                      # step k-1's results are on the host
            readback[1 - b].synchronize()
            _ = float(hl[1 - b][0])
    readback[(args.steps - 1) % 2].synchronize()
    _ = float(hl[(args.steps - 1) % 2][0])
    e2e_pipe_s = time.perf_counter() - t0
    wl.check()
    wl.verts, wl.tex, wl.targets, wl.sid, wl.gt, wl.gv, wl.loss = home
    e2e_pipe_s = max_over_ranks(e2e_pipe_s, world, dev)
    barrier()

    extras = {}
    if not args.views and not args.no_extras:
        extras["plain_path"] = _plain_leg(wl, max(2, args.steps // 2))
    if rank != 0:
        return None
    frags_total = wl.fragments * args.steps * world
    value = whole_job_value(wl.fragments, args.steps, world, t_max)
    peak, peak_kind = _peaks()
    algo = wl.algorithmic_bytes()
    stage_ms = {k: v[1] for k, v in prof.items() if v[0] > 0}
    dom = max((k for k in stage_ms if k in algo), key=lambda k: stage_ms[k])
    runs = prof[dom][0]
    per_launch_ms = prof[dom][1] / runs
    achieved = algo[dom] / (per_launch_ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded soups, cameras, targets)",
        "config": workload_config(world),
        "workload_stats": {"fragments_per_step": wl.fragments, "bin_pairs": wl.pairs, "tuning": tuning},
        "ms_per_step_dist": {"mean": ms / args.steps, "median": float(np.median(step_ms)),
                             "p10": float(np.percentile(step_ms, 10)), "p90": float(np.percentile(step_ms, 90)),
                             "min": float(min(step_ms)), "max": float(max(step_ms)),
                             "what": "one CUDA event pair per timed step (rank 0)"},
        "e2e": {"value": frags_total / e2e_serial_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "what": "serial: inputs copied in, the step, texture and vertex gradients and the loss copied "
                        "out, host waits; nothing overlaps"},
        "e2e_pipelined": {"value": frags_total / e2e_pipe_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                          "d2h_bytes_per_step": d2h,
                          "what": "the same copies double buffered: inputs of step k+1 and gradients of step k "
                                  "move on two copy streams while the next step computes"},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": _traffic(dom, wl.pixel_samples),
                     "algorithmic_bytes": algo[dom], "launch_ms": per_launch_ms,
                     "step_bytes": wl.step_bytes(),
                     "step_frac": wl.step_bytes() / (t_max / args.steps / 1e3) / 1e9 / peak,
                     "counters": _counters(dom)},
        "stages_ms_per_step": {k: v / args.steps for k, v in stage_ms.items()},
        "clocks": clk.summary(),
    }
    if extras:
        line["plain_path"] = extras["plain_path"]
        line["plain_path"]["batched_speedup"] = value / world / extras["plain_path"]["value"]
    if not args.views and not args.no_extras and world == 1:
        for name in ("plain_small", "batched_views"):
            leg = _config_leg(name, dev, 200 if name == "plain_small" else 50)
            if not args.no_cpu_baseline:
                leg["cpu_oracle"] = _config_cpu(name, leg["views"])
            line[name] = leg
        line["shade"] = _shade_leg(wl, max(5, args.steps // 4))
        line["adapt"] = _adapt_leg(wl)
        line["loss_optim"] = _loss_optim_leg(wl)
        del wl
        torch.cuda.empty_cache()
        line["levels"] = _levels_leg(dev, max(5, args.steps // 4))
        torch.cuda.empty_cache()
        line["paper_step"] = _paper_step_leg(dev, max(5, args.steps // 4))
        torch.cuda.empty_cache()
        line["train"] = _train_leg(dev, args.train_iters)
        torch.cuda.empty_cache()
        if args.serve_seconds > 0:
            line["serve"] = _serve_leg(dev, args.serve_seconds, plain=False)
            line["serve_plain"] = _serve_leg(dev, args.serve_seconds, plain=True)
            line["serve_sweep"] = _serve_sweep(dev)
    return line


# ---------------------------------------------------------------- CPU oracle
# The CPU baseline times the oracle in its bbox-scan (object-order) mode,
# whose results equal the brute-force oracle's bit for bit, on bands of rows
# of the workload's first view (1920x1080, S = 4, forward + L2 loss +
# backward with every gradient term); the targets of those rows are rendered
# beforehand, untimed.  Both the cpu_baseline of the GPU arm and the
# reference arm time this same sample: rows ROW0, ROW0 + 1, ... of view 0,
# one row per process.
_ORACLE_SCENES = {}
CPU_VIEW = 0
CPU_ROW0 = 400


def _oracle_init():
    """Pool initializer: each worker builds the workload and target soups once
    (not timed)."""
    import oracle as O
    O.build()
    _ORACLE_SCENES["sc"] = I.large_batch()
    _ORACLE_SCENES["tsc"] = I.large_batch(soup_seed=12)


def _oracle_target(job):
    """Untimed: the target colours [C-1, r1-r0, W] of rows [r0, r1) of a view
    (the target soup's binary-opacity render, Eq. 3)."""
    import oracle as O
    if not _ORACLE_SCENES:
        _oracle_init()
    view, r0, r1 = job
    sc, tsc = _ORACLE_SCENES["sc"], _ORACLE_SCENES["tsc"]
    tg = O.forward(tsc.verts, tsc.tex, tsc.grid_n, [sc.cams[view]], np.zeros(1, np.uint64), S=1,
                   mode=O.MODE_THRESHOLD_HALF, bg=sc.bg, rows=(r0, r1), scan=True)[0]
    return tg["color"][0][:, r0:r1].copy()


def _oracle_rows(job):
    """One timed unit: forward + L2 loss + backward of the oracle (bbox-scan
    mode) on rows [r0, r1) of one view against precomputed target rows.
    Returns (fragments, seconds)."""
    import oracle as O
    if not _ORACLE_SCENES:
        _oracle_init()
    view, r0, r1, seed, tgt = job
    sc = _ORACLE_SCENES["sc"]
    cam = sc.cams[view]
    S = sc.samples
    t0 = time.perf_counter()
    f = O.forward(sc.verts, sc.tex, sc.grid_n, [cam], np.array([seed], np.uint64), S=S, bg=sc.bg,
                  rows=(r0, r1), scan=True)[0]
    d = f["color"][:, :, r0:r1] - tgt[None]                     # the band only
    gc = np.zeros(f["color"].shape, np.float32)
    gc[:, :, r0:r1] = 2.0 * d / S
    sw = np.zeros(f["tri_id"].shape, np.float32)
    sw[:, r0:r1] = (d.astype(np.float64) ** 2).sum(1) / S
    O.backward(sc.verts, sc.tex, sc.grid_n, [cam], S, [f], [gc], [sw], rows=(r0, r1), scan=True)
    frags = int(f["n_cover"][:, r0:r1].sum())
    return frags, time.perf_counter() - t0


def _cores():
    n = os.cpu_count() or 1
    return max(1, min(16, n))


def oracle_pool(cores: int):
    """A spawned pool (never forked after a GPU call) whose workers hold the
    workload."""
    return mp.get_context("spawn").Pool(cores, initializer=_oracle_init)


def oracle_sample(pool, cores: int, start_row: int, seed: int = 13, rows_per_process: int = 1):
    """Rows start_row .. start_row + cores * rows_per_process - 1 of view
    CPU_VIEW, one band of rows_per_process rows per process; fragments/s over
    the wall time of the timed pass (targets rendered before, untimed)."""
    n = rows_per_process
    rows = [(CPU_VIEW, start_row + n * k, start_row + n * (k + 1)) for k in range(cores)]
    tg = pool.map(_oracle_target, rows)
    jobs = [r + (seed, t) for r, t in zip(rows, tg)]
    t0 = time.perf_counter()
    res = pool.map(_oracle_rows, jobs)
    wall = time.perf_counter() - t0
    frags = sum(r[0] for r in res)
    return frags / wall, wall, frags


def oracle_one_core(start_row: int, n_rows: int, seed: int = 13):
    """The unit of one process of oracle_sample on one core, in this process:
    the band of rows start_row .. start_row + n_rows - 1 in one call (the
    oracle's per-call candidate scan is paid once per band, as there)."""
    r = (CPU_VIEW, start_row, start_row + n_rows)
    tg = _oracle_target(r)
    frags, secs = _oracle_rows(r + (seed, tg))
    return frags / secs, secs, frags


def _train_cpu_job(job):
    """CPU oracle (bbox-scan mode) on rows [r0, r1) of one training view
    (20,000 triangles, 1024x768, S = 1): forward + L2 loss + backward against
    the reference soup's render of those rows (rendered first, untimed).
    Returns seconds."""
    import oracle as O
    r0, r1 = job
    if "train" not in _ORACLE_SCENES:
        _ORACLE_SCENES["train"] = I.training_setup()
    sc, ref = _ORACLE_SCENES["train"]
    cam = sc.cams[0]
    tg = O.forward(ref.verts, ref.tex, ref.grid_n, [cam], np.zeros(1, np.uint64), S=1,
                   mode=O.MODE_THRESHOLD_HALF, bg=sc.bg, rows=(r0, r1), scan=True)[0]["color"][0][:, r0:r1]
    t0 = time.perf_counter()
    f = O.forward(sc.verts, sc.tex, sc.grid_n, [cam], np.array([9], np.uint64), S=1, bg=sc.bg, rows=(r0, r1),
                  scan=True)[0]
    d = f["color"][:, :, r0:r1] - tg[None]
    gc = np.zeros(f["color"].shape, np.float32)
    gc[:, :, r0:r1] = 2.0 * d
    sw = np.zeros(f["tri_id"].shape, np.float32)
    sw[:, r0:r1] = (d.astype(np.float64) ** 2).sum(1)
    O.backward(sc.verts, sc.tex, sc.grid_n, [cam], 1, [f], [gc], [sw], rows=(r0, r1), scan=True)
    return time.perf_counter() - t0


def _serve_cpu_job(job):
    """CPU oracle forward (bbox-scan mode, binary opacity, S = 1) of rows
    [r0, r1) of one served request.  Returns (seconds, rows of the frame)."""
    import oracle as O
    k, cam, seed, r0, r1 = job
    if "serve" not in _ORACLE_SCENES:
        _ORACLE_SCENES["serve"] = I.serving_workload(duration=0.0)[0]
    sc = _ORACLE_SCENES["serve"][k]
    t0 = time.perf_counter()
    O.forward(sc.verts, sc.tex, sc.grid_n, [cam], np.array([seed], np.uint64), S=1, mode=O.MODE_THRESHOLD_HALF,
              bg=sc.bg, rows=(r0, r1), scan=True)
    return time.perf_counter() - t0, cam.height


def cpu_config_estimates():
    """The oracle on the training step and on the serving stream, extrapolated
    from bounded samples (marked "extrapolated"): one row band per process."""
    cores = _cores()
    with mp.get_context("spawn").Pool(cores) as pool:
        bands = [(300 + 2 * k, 302 + 2 * k) for k in range(cores)]
        secs = pool.map(_train_cpu_job, bands)
        s_per_row = float(np.mean(secs)) / 2
        rows_per_step = 4 * 768
        train = {"iters_per_s": 1.0 / (s_per_row * rows_per_step / cores), "cores": cores,
                 "iters_per_s_cores_1": 1.0 / (s_per_row * rows_per_step),
                 "kind": "oracle (bbox-scan mode), extrapolated",
                 "sample": "%d bands of 2 rows of a 1024x768 training view, forward + L2 + backward, S=1" % cores}
        _, reqs = I.serving_workload(duration=0.05, arrival_seed=40)
        jobs = []
        for i, (_, k, cam, seed) in enumerate(reqs[:2 * cores]):
            r0 = cam.height // 2
            jobs.append((k, cam, seed, r0, r0 + 2))
        res = pool.map(_serve_cpu_job, jobs)
        frame_s = float(np.mean([t / 2 * h for t, h in res]))
        serve = {"frames_per_s": cores / frame_s, "cores": cores, "frames_per_s_cores_1": 1.0 / frame_s,
                 "kind": "oracle (bbox-scan mode), extrapolated",
                 "sample": "2 middle rows of each of %d requests of the stream (frames of 256x256 .. 1920x1080), "
                           "forward with binary opacity" % len(jobs)}
    return {"train": train, "serve": serve}


# Rows per process of the CPU baseline's sample (about 10-20 s of CPU work
# in all on 16 cores) and of each step of the reference arm.
CPU_ROWS_BASELINE = 40
CPU_ROWS_STEP = 4


def cpu_baseline_entry(fragments_per_step=None):
    cores = _cores()
    n = CPU_ROWS_BASELINE
    with oracle_pool(cores) as pool:
        v, wall, frags = oracle_sample(pool, cores, CPU_ROW0, rows_per_process=n)
    v1, secs1, frags1 = oracle_one_core(CPU_ROW0, n)
    out = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle (bbox-scan mode, results equal to brute force)",
           "sample": "rows %d-%d of view %d (1920x1080), %d rows per process, S=4, forward + L2 loss + backward "
                     "(all gradient terms), targets rendered before, untimed: %d fragments in %.2f s wall"
                     % (CPU_ROW0, CPU_ROW0 + n * cores - 1, CPU_VIEW, n, frags, wall),
           "cores_1": {"value": v1, "unit": UNIT, "cores": 1,
                       "sample": "rows %d-%d of the same view on one core: %d fragments in %.2f s"
                                 % (CPU_ROW0, CPU_ROW0 + n - 1, frags1, secs1)}}
    if fragments_per_step:
        out["extrapolated_s_per_step"] = {"cores": fragments_per_step / v, "cores_1": fragments_per_step / v1,
                                          "what": "extrapolated: the step's fragments at the sampled rate"}
    return out


def _reference_arm(args):
    world, rank, _ = _dist()
    if rank != 0:
        return None
    cores = _cores()
    for _ in range(args.warmup):
        pass   # the oracle has no warm-up state; warm-up samples would only repeat the work
    # each step: the next band of rows of the workload's first view, one row
    # per process (the rows the GPU arm's cpu_baseline times come first)
    vals, walls, total = [], [], 0
    n = CPU_ROWS_STEP
    with oracle_pool(cores) as pool:
        for k in range(args.steps):
            start = CPU_ROW0 + (n * cores * k) % (1080 - CPU_ROW0 - n * cores)
            v, wall, frags = oracle_sample(pool, cores, start_row=start, rows_per_process=n)
            vals.append(v)
            walls.append(wall)
            total += frags
    value = total / sum(walls)
    sample = ("per step %d rows of view %d (1920x1080), %d rows per process, from row %d on, S=4, forward + L2 "
              "loss + backward; oracle in bbox-scan mode" % (n * cores, CPU_VIEW, n, CPU_ROW0))
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded soups, cameras, targets)",
            "config": workload_config(world),
            "impl": "reference",
            "cpu_baseline": {"kind": "oracle (bbox-scan mode)", "cores": cores, "value": value, "unit": UNIT,
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--views", type=int, default=0,
                    help="use only the first N views (reduced case for profiler captures; not a bench line)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the plain-path, training-step and serving legs")
    ap.add_argument("--train-iters", type=int, default=50)
    ap.add_argument("--no-tune", action="store_true", help="default launch parameters instead of the autotuner's")
    ap.add_argument("--unfused", action="store_true",
                    help="separate forward, loss and backward calls instead of the fused training pass")
    ap.add_argument("--tuning", default="", help="fixed launch parameters tile_w,depth_bits,blocks_per_sm,chunk")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--widened-cases", action="store_true",
                    help="one launch of each widened-row kernel (profiler captures; not a bench line)")
    args = ap.parse_args()
    if args.widened_cases:
        widened_cases()
        return
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    if args.impl == "reference":
        line = _reference_arm(args)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    world, rank, _ = _dist()
    cpu = None
    cpu_est = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.views:
        cpu = cpu_baseline_entry()   # before the first GPU call (spawned workers)
        if not args.no_extras:
            cpu_est = cpu_config_estimates()
    line = _gpu_arm(args)
    if line is not None:
        if cpu is not None:
            f = line["workload_stats"]["fragments_per_step"]
            cpu["extrapolated_s_per_step"] = {"cores": f / cpu["value"], "cores_1": f / cpu["cores_1"]["value"],
                                              "what": "extrapolated: the step's fragments at the sampled rate"}
        line["cpu_baseline"] = cpu
        if cpu_est is not None:
            if "train" in line:
                line["train"]["cpu_oracle"] = cpu_est["train"]
            if "serve" in line:
                line["serve"]["cpu_oracle"] = cpu_est["serve"]
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
