"""Multi-resolution texture helpers (Sec. 3.3; supplementary
"Coarse-to-Fine Optimization") over ``ds_levels_*``.

A multi-resolution texture is one flat float32 CUDA tensor holding levels
r_min..r_max back to back, level R as [T, V_R, C] (V_R = (2^R+1)(2^R+2)/2);
``Context.soup_upload_levels`` registers it, and every pass then renders the
sum of the levels on the finest grid and returns gradients per level.
"""
from __future__ import annotations

import torch

from . import native as N


def zeros(T: int, r_min: int, r_max: int, C: int, device="cuda") -> torch.Tensor:
    """All-zero level logits (the paper's initialisation: features 0.5 after the sigmoid)."""
    return torch.zeros(sum(N.level_sizes(T, r_min, r_max, C)), dtype=torch.float32, device=device)


def compose(tex_levels: torch.Tensor, T: int, r_min: int, r_max: int, C: int, activate: bool = True):
    """The finest grid [T, V_{r_max}, C]: sigmoid of the composed logits (the
    texture kept after training) or the logits themselves."""
    out = torch.empty((T, N.level_V(r_max), C), dtype=torch.float32, device=tex_levels.device)
    N.levels_compose(tex_levels, T, r_min, r_max, C, out, activate=activate)
    return out


def coarse_to_fine(coarse: torch.Tensor, r_coarse: int, r_min: int, r_max: int, reset_alpha: bool = True):
    """The switch from the coarse stage to levels r_min..r_max: the coarse
    grid's features ([T, V_{r_coarse}, C] logits) are sampled at the vertices
    of level r_min and copied there, the other levels start at zero, and the
    opacity channel (the last) is re-initialised to zero logits in every
    level.  Returns the flat level tensor."""
    T, _, C = coarse.shape
    out = zeros(T, r_min, r_max, C, coarse.device)
    first = N.split_levels(out, T, r_min, r_max, C)[0]
    N.levels_resample(coarse.contiguous(), T, r_coarse, C, first, r_min)
    if reset_alpha:
        first[:, :, C - 1] = 0.0
    return out
