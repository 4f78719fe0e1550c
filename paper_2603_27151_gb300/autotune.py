"""Autotuned launch parameters with a persistent cache.

``tuned(ctx, ...)`` looks the workload up in a JSON cache (key: device name,
triangle count, grid size N, channels C, samples S, mode, whether the
backward is timed, and the sorted view resolutions); on a miss it runs the
library's autotuner (``ds_autotune``: coordinate search over tile shape,
depth bits of the bin key, staging chunk and CTAs per SM, each candidate timed
with CUDA events) and stores the result.  The tuning is set on the context
either way.  Cache file: ``$DS_TUNE_CACHE`` or
``~/.cache/diffsoup/tuning.json``.
"""
from __future__ import annotations

import json
import os

from . import native as N


def cache_path() -> str:
    return os.environ.get("DS_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "diffsoup", "tuning.json"))


def workload_key(device_name: str, T: int, grid_n: int, C: int, S: int, mode: int, backward: bool, cams) -> str:
    res = sorted("%dx%d" % (c.width, c.height) for c in cams)
    return "|".join([device_name, "T%d" % T, "N%d" % grid_n, "C%d" % C, "S%d" % S, "m%d" % mode,
                     "bwd" if backward else "fwd", ",".join(res)])


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, table: dict):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuned(ctx: "N.Context", soup_id: int, T: int, grid_n: int, C: int, cams, seeds, S: int, mode: int, bg,
          gbufs, colors, grad_colors=None, score_ws=None, grad_verts=None, grad_tex=None, reps: int = 3,
          path: str | None = None, device_name: str | None = None, targets=None, scale: float = 1.0) -> dict:
    """The cached (or freshly tuned) tuning of this workload, set on ``ctx``.
    With ``targets`` the fused training pass is what is timed."""
    import torch
    path = path or cache_path()
    name = device_name or torch.cuda.get_device_name(ctx.device)
    key = workload_key(name, T, grid_n, C, S, mode, grad_colors is not None, cams)
    if targets is not None:
        key += "|fusedL2"
    table = _load(path)
    hit = table.get(key)
    if hit is not None:
        ctx.set_tuning(hit["tile_w"], hit["depth_bits"], hit["blocks_per_sm"], hit["chunk"])
        return dict(hit, cached=True)
    best, ms = ctx.autotune(soup_id, cams, seeds, S, mode, bg, gbufs, colors, grad_colors, score_ws, grad_verts,
                            grad_tex, reps=reps, targets=targets, scale=scale)
    table = _load(path)
    table[key] = dict(best, ms=ms)
    _store(path, table)
    return dict(best, ms=ms, cached=False)
