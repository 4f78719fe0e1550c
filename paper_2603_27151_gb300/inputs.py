"""Seeded synthetic inputs: triangle soups, texture logits, pinhole cameras, seeds.

This module only draws inputs.  It holds none of the rasterisation method's
arithmetic (no projection, coverage, masking, texture decode or gradient), so
both the CUDA path and the CPU oracle can consume what it produces.

Soups follow the paper's random soup initialisation (supplementary "Random
Triangle Soup Initialization"): seed points uniform in a box, one triangle of
random orientation around each point.  Texture logits are i.i.d. N(0, 1), so
the activated opacity has mean 0.5 and masking is heavy.  Cameras are pinholes
on a sphere looking at the origin, 45 degree vertical field of view.

Camera convention (shared by every consumer): world -> camera is
``x_c = R @ v + t``; +z is forward, +x right, +y down; pixel (px, py) has its
centre at (px + 0.5, py + 0.5); ``fx = fy = H / (2 tan(fov / 2))``,
``cx = W / 2``, ``cy = H / 2``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def n_texels(grid_n: int) -> int:
    """Feature vertices of a triangle subdivided ``grid_n`` times per edge."""
    return (grid_n + 1) * (grid_n + 2) // 2


@dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray          # (3, 3) float32, world -> camera rotation (rows: right, down, forward)
    t: np.ndarray          # (3,) float32
    near: float = 0.01

    def as_floats(self) -> np.ndarray:
        """(fx, fy, cx, cy, R row-major, t, near) as 17 float32 values."""
        return np.concatenate([
            np.array([self.fx, self.fy, self.cx, self.cy], np.float32),
            self.R.astype(np.float32).reshape(9),
            self.t.astype(np.float32).reshape(3),
            np.array([self.near], np.float32),
        ]).astype(np.float32)


@dataclass
class Scene:
    verts: np.ndarray              # (T, 3, 3) float32
    tex: np.ndarray                # (T, V, C) float32 logits; channel C-1 is opacity
    grid_n: int
    cams: list = field(default_factory=list)
    seeds: np.ndarray = None       # (n_views,) uint64 mask seeds
    samples: int = 1
    bg: np.ndarray = None          # (C-1,) float32

    @property
    def T(self) -> int:
        return int(self.verts.shape[0])

    @property
    def C(self) -> int:
        return int(self.tex.shape[2])


def look_at(eye, width: int, height: int, fov_deg: float = 45.0, near: float = 0.01) -> Camera:
    eye = np.asarray(eye, np.float64)
    fwd = -eye / np.linalg.norm(eye)
    up = np.array([0.0, 0.0, 1.0])
    if abs(float(fwd @ up)) > 0.99:
        up = np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    t = -R @ eye
    f = height / (2.0 * math.tan(math.radians(fov_deg) / 2.0))
    return Camera(width, height, float(np.float32(f)), float(np.float32(f)),
                  width / 2.0, height / 2.0, R.astype(np.float32), t.astype(np.float32), near)


def sphere_eyes(n: int, radius: float, rng: np.random.Generator) -> np.ndarray:
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d * radius


def iid_soup(T: int, rng: np.random.Generator) -> np.ndarray:
    """Every vertex i.i.d. uniform in [-1, 1]^3 (independent triangles)."""
    return rng.uniform(-1.0, 1.0, (T, 3, 3)).astype(np.float32)


def edge_length_for(T: int) -> float:
    """Edge length that keeps the total soup area of 2,000 triangles of edge 0.2."""
    return 0.2 * math.sqrt(2000.0 / T)


def box_soup(T: int, edge: float, rng: np.random.Generator, half: float = 1.0) -> np.ndarray:
    """Equilateral triangles of edge ``edge``, centres uniform in [-half, half]^3,
    random unit normal and random in-plane angle."""
    c = rng.uniform(-half, half, (T, 3))
    n = rng.standard_normal((T, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    a = rng.standard_normal((T, 3))
    u = a - (a * n).sum(1, keepdims=True) * n
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    w = np.cross(n, u)
    phi = rng.uniform(0.0, 2.0 * math.pi, T)
    r = edge / math.sqrt(3.0)
    out = np.empty((T, 3, 3))
    for i in range(3):
        ang = phi + 2.0 * math.pi * i / 3.0
        out[:, i, :] = c + r * (np.cos(ang)[:, None] * u + np.sin(ang)[:, None] * w)
    return out.astype(np.float32)


def logits(T: int, grid_n: int, C: int, rng: np.random.Generator) -> np.ndarray:
    return rng.standard_normal((T, n_texels(grid_n), C)).astype(np.float32)


def level_logits(T: int, r_min: int, r_max: int, C: int, rng: np.random.Generator) -> list:
    """Multi-resolution logits: level R (2^R subdivisions) as [T, V_R, C],
    normal with standard deviation 1/sqrt(number of levels)."""
    sd = 1.0 / math.sqrt(r_max - r_min + 1)
    return [(sd * rng.standard_normal((T, n_texels(1 << R), C))).astype(np.float32) for R in range(r_min, r_max + 1)]


def levels_scene(soup_seed: int = 21, cam_seed: int = 22, mask_seed: int = 23, T: int = 2000,
                 r_min: int = 2, r_max: int = 5, res=((128, 128), (256, 192), (97, 61))):
    """(Scene with the composed-texture shape, level logits): 2,000 triangles of
    edge 0.2, 8 channels, levels r_min..r_max, views at mixed resolutions."""
    rng = np.random.default_rng(soup_seed)
    verts = box_soup(T, 0.2, rng)
    lv = level_logits(T, r_min, r_max, 8, rng)
    eyes = sphere_eyes(len(res), 3.0, np.random.default_rng(cam_seed))
    cams = [look_at(e, w, h) for e, (w, h) in zip(eyes, res)]
    sc = Scene(verts, np.zeros((T, n_texels(1 << r_max), 8), np.float32), 1 << r_max, cams,
               mask_seeds(mask_seed, len(res)), 1, np.zeros(7, np.float32))
    return sc, lv


def mask_seeds(seed: int, n: int) -> np.ndarray:
    return np.random.SeedSequence(seed).generate_state(n, dtype=np.uint64)


# ----------------------------------------------------------------------------
# The five workloads (sizes, seeds and distributions are fixed here)
# ----------------------------------------------------------------------------

def plain_small(soup_seed: int = 0, mask_seed: int = 0) -> Scene:
    """64 triangles with i.i.d. vertices, N=4 grid, RGB + opacity, one 64x64 view."""
    rng = np.random.default_rng(soup_seed)
    verts = iid_soup(64, rng)
    tex = logits(64, 4, 4, rng)
    cam = look_at([0.0, 0.0, 3.0], 64, 64)
    return Scene(verts, tex, 4, [cam], mask_seeds(mask_seed, 1), 1, np.zeros(3, np.float32))


def batched_views(soup_seed: int = 2, cam_seed: int = 3, mask_seed: int = 5) -> Scene:
    """2,000 triangles of edge 0.2, N=8, 8 channels, 8 views at mixed resolutions."""
    rng = np.random.default_rng(soup_seed)
    verts = box_soup(2000, 0.2, rng)
    tex = logits(2000, 8, 8, rng)
    eyes = sphere_eyes(8, 3.0, np.random.default_rng(cam_seed))
    res = [(128, 128)] * 3 + [(256, 256)] * 3 + [(320, 240)] * 2
    cams = [look_at(e, w, h) for e, (w, h) in zip(eyes, res)]
    return Scene(verts, tex, 8, cams, mask_seeds(mask_seed, 8), 1, np.zeros(7, np.float32))


def large_batch(soup_seed: int = 10, cam_seed: int = 11, mask_seed: int = 13,
                T: int = 100_000, samples: int = 4) -> Scene:
    """100,000 triangles, N=8, 8 channels; 4 views at 1920x1080 + 4 at 960x540, 4 mask samples."""
    rng = np.random.default_rng(soup_seed)
    verts = box_soup(T, edge_length_for(T), rng)
    tex = logits(T, 8, 8, rng)
    eyes = sphere_eyes(8, 3.0, np.random.default_rng(cam_seed))
    res = [(1920, 1080)] * 4 + [(960, 540)] * 4
    cams = [look_at(e, w, h) for e, (w, h) in zip(eyes, res)]
    return Scene(verts, tex, 8, cams, mask_seeds(mask_seed, 8), samples, np.zeros(7, np.float32))


def training_setup(soup_seed: int = 6, ref_seed: int = 7, cam_seed: int = 8,
                   T: int = 20_000, T_ref: int = 200_000, n_cams: int = 100,
                   width: int = 1024, height: int = 768):
    """Training soup (20k triangles), reference soup (200k) and 100 cameras at 1024x768."""
    rng = np.random.default_rng(soup_seed)
    verts = box_soup(T, edge_length_for(T), rng)
    tex = logits(T, 8, 8, rng)
    rr = np.random.default_rng(ref_seed)
    ref_verts = box_soup(T_ref, edge_length_for(T_ref), rr)
    ref_tex = logits(T_ref, 8, 8, rr)
    eyes = sphere_eyes(n_cams, 3.0, np.random.default_rng(cam_seed))
    cams = [look_at(e, width, height) for e in eyes]
    return (Scene(verts, tex, 8, cams, None, 1, np.zeros(7, np.float32)),
            Scene(ref_verts, ref_tex, 8, cams, None, 1, np.zeros(7, np.float32)))


def step_views(step: int, n_cams: int = 100, per_step: int = 4, base_seed: int = 9):
    """Camera indices and mask seeds for one training step (4 views per step)."""
    ss = np.random.SeedSequence([base_seed, step])
    rng = np.random.default_rng(ss)
    idx = rng.choice(n_cams, per_step, replace=False)
    seeds = ss.spawn(1)[0].generate_state(per_step, dtype=np.uint64)
    return idx, seeds


SERVE_RESOLUTIONS = [(256, 256), (640, 480), (1280, 720), (1920, 1080)]


def serving_workload(n_soups: int = 16, rate: float = 2000.0, duration: float = 10.0,
                     soup_seed0: int = 20, arrival_seed: int = 40):
    """16 soups with log-uniform triangle counts in [5000, 50000] and a Poisson
    request stream (arrival time, soup index, camera, seed)."""
    soups = []
    for i in range(n_soups):
        rng = np.random.default_rng(soup_seed0 + i)
        T = int(math.floor(math.exp(rng.uniform(math.log(5000), math.log(50000)))))
        soups.append(Scene(box_soup(T, edge_length_for(T), rng), logits(T, 8, 8, rng), 8,
                           [], None, 1, np.zeros(7, np.float32)))
    rng = np.random.default_rng(arrival_seed)
    n = rng.poisson(rate * duration)
    times = np.sort(rng.uniform(0.0, duration, n))
    which = rng.integers(0, n_soups, n)
    res = rng.integers(0, len(SERVE_RESOLUTIONS), n)
    eyes = sphere_eyes(n, 3.0, rng)
    seeds = rng.integers(0, 2**63, n, dtype=np.uint64)
    reqs = [(float(times[i]), int(which[i]), look_at(eyes[i], *SERVE_RESOLUTIONS[res[i]]), int(seeds[i]))
            for i in range(n)]
    return soups, reqs
