"""CPU oracle for the DiffSoup hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it.

``build()`` compiles ``diffsoup_oracle.c`` with gcc into ``oracle/_build``;
the wrappers below marshal numpy arrays into it.  See the C file for the
passage of the paper that each function restates and for its pin status.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "diffsoup_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")

MODE_STOCHASTIC = 0
MODE_THRESHOLD_HALF = 1
G_TEX, G_SCORE, G_INTERIOR, G_EDGE = 1, 2, 4, 8
G_ALL = G_TEX | G_SCORE | G_INTERIOR | G_EDGE

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, no fused multiply-add contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_OUT)
        f32, i32, u32, i64, u64 = ctypes.c_float, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64
        P = ctypes.c_void_p
        L.or_expf.restype = f32; L.or_expf.argtypes = [f32]
        L.or_sigmoidf.restype = f32; L.or_sigmoidf.argtypes = [f32]
        L.or_philox4x32.restype = None; L.or_philox4x32.argtypes = [P, P, P]
        L.or_tau.restype = f32; L.or_tau.argtypes = [u64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.or_lookup.restype = f32; L.or_lookup.argtypes = [P, ctypes.c_int, ctypes.c_int, f32, f32]
        L.or_cell.restype = None; L.or_cell.argtypes = [ctypes.c_int, f32, f32, P, P]
        L.or_fragment.restype = ctypes.c_int
        L.or_fragment.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
        L.or_activate.restype = None; L.or_activate.argtypes = [P, i64, P]
        L.or_forward.restype = ctypes.c_int
        L.or_forward.argtypes = [P, P, i32, i32, i32, P, P, P, i32, i32, i32, P, P, i32, i32,
                                 P, P, P, P, P, P, i32]
        L.or_backward.restype = ctypes.c_int
        L.or_backward.argtypes = [P, P, i32, i32, i32, P, P, i32, i32, P, P, P, P, P, u32, i32, i32, P, P, i32]
        L.or_compose.restype = None; L.or_compose.argtypes = [P, i32, i32, i32, i32, P]
        L.or_coverage.restype = None; L.or_coverage.argtypes = [P, i64, i32, P]
        L.or_edge_ratios.restype = None; L.or_edge_ratios.argtypes = [P, i32, P, P, i32, P]
        L.or_soup_rebuild.restype = None
        L.or_soup_rebuild.argtypes = [P, P, i32, i32, i32, i32, P, i32, P, P]
        L.or_restrict.restype = None; L.or_restrict.argtypes = [P, i32, i32, i32, i32, P]
        L.or_resample.restype = None; L.or_resample.argtypes = [P, i32, i32, i32, P, i32]
        L.or_expected.restype = ctypes.c_int
        L.or_expected.argtypes = [P, P, i32, i32, i32, P, P, i32, P, P, P, P]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _cams(cams):
    cf = np.stack([c.as_floats() for c in cams]).astype(np.float32)
    wh = np.array([[c.width, c.height] for c in cams], np.int32)
    return np.ascontiguousarray(cf), np.ascontiguousarray(wh)


# ---------------------------------------------------------------- scalar pins
def expf(x: float) -> float:
    return float(lib().or_expf(float(x)))


def sigmoidf(x: float) -> float:
    return float(lib().or_sigmoidf(float(x)))


def philox(ctr, key) -> np.ndarray:
    c = _c(ctr, np.uint32); k = _c(key, np.uint32); out = np.zeros(4, np.uint32)
    lib().or_philox4x32(_p(c), _p(k), _p(out))
    return out


def tau(seed: int, px: int, py: int, t: int, s: int) -> float:
    return float(lib().or_tau(int(seed), px, py, t, s))


def lookup(grid: np.ndarray, N: int, b1: float, b2: float) -> float:
    """Value of a single-channel grid (V,) at (b1, b2)."""
    g = _c(grid, np.float32)
    return float(lib().or_lookup(_p(g), N, 1, float(b1), float(b2)))


def cell(N: int, b1: float, b2: float):
    idx = np.zeros(3, np.int32); w = np.zeros(2, np.float32)
    lib().or_cell(N, float(b1), float(b2), _p(idx), _p(w))
    return idx, w


def fragment(v9, cam, px: int, py: int):
    """(covered, rho, D, b1, b2) of one triangle at one pixel."""
    v = _c(v9, np.float32).reshape(9); cf = cam.as_floats(); out = np.zeros(4, np.float32)
    cov = lib().or_fragment(_p(v), _p(cf), cam.width, cam.height, px, py, _p(out))
    return bool(cov), float(out[0]), float(out[1]), float(out[2]), float(out[3])


def activate(tex: np.ndarray) -> np.ndarray:
    t = _c(tex, np.float32); out = np.empty_like(t)
    lib().or_activate(_p(t), t.size, _p(out))
    return out


# ------------------------------------------------------- multi-resolution
def level_V(R: int) -> int:
    n = 1 << R
    return (n + 1) * (n + 2) // 2


def compose(levels, r_min: int, r_max: int) -> np.ndarray:
    """Composed logits [T, V_f, C] of the finest grid from the level grids
    ``levels[k]`` = level r_min + k, [T, V_R, C] (FP32, see or_compose)."""
    T, _, C = levels[0].shape
    flat = np.concatenate([_c(l, np.float32).reshape(-1) for l in levels])
    out = np.empty((T, level_V(r_max), C), np.float32)
    lib().or_compose(_p(flat), T, r_min, r_max, C, _p(out))
    return out


def restrict(gfine, r_min: int, r_max: int):
    """Per-level gradients (FP64) given the gradient of the composed logits."""
    g = _c(gfine, np.float64)
    T, _, C = g.shape
    sizes = [T * level_V(R) * C for R in range(r_min, r_max + 1)]
    out = np.empty(sum(sizes), np.float64)
    lib().or_restrict(_p(g), T, r_min, r_max, C, _p(out))
    parts, o = [], 0
    for R, n in zip(range(r_min, r_max + 1), sizes):
        parts.append(out[o:o + n].reshape(T, level_V(R), C))
        o += n
    return parts


def resample(src, r_src: int, r_dst: int) -> np.ndarray:
    s = _c(src, np.float32)
    T, _, C = s.shape
    out = np.empty((T, level_V(r_dst), C), np.float32)
    lib().or_resample(_p(s), T, r_src, C, _p(out), r_dst)
    return out


def forward_levels(verts, levels, r_min: int, r_max: int, cams, seeds, S=1, mode=MODE_STOCHASTIC, bg=None):
    """Forward of a soup whose texture is the composition of level grids."""
    return forward(verts, compose(levels, r_min, r_max), 1 << r_max, cams, seeds, S=S, mode=mode, bg=bg)


def backward_levels(verts, levels, r_min: int, r_max: int, cams, S, fwd, grad_color, score_w, flags=G_ALL):
    """(per-level texture gradients, vertex gradient) of a level soup: the
    fine-grid backward followed by the adjoint of the composition."""
    gt, gv = backward(verts, compose(levels, r_min, r_max), 1 << r_max, cams, S, fwd, grad_color, score_w,
                      flags=flags)
    return restrict(gt, r_min, r_max), gv


# ------------------------------------------------------- adaptive control
def coverage(tri_ids, T: int) -> np.ndarray:
    """Pixel-samples selected per triangle (int64 [T]) of tri_id planes."""
    counts = np.zeros(T, np.int64)
    for a in tri_ids:
        a = _c(a, np.int32)
        lib().or_coverage(_p(a), a.size, T, _p(counts))
    return counts


def edge_ratios(verts, cams) -> np.ndarray:
    """[T, 3] largest view-space edge length / image height over the views."""
    v = _c(verts, np.float32)
    cf, wh = _cams(cams)
    out = np.zeros((v.shape[0], 3), np.float32)
    lib().or_edge_ratios(_p(v), v.shape[0], _p(cf), _p(wh), len(cams), _p(out))
    return out


def adapt_plan(counts, ratios, threshold: float, budget: int):
    """One round of adaptive control (Sec. 3.4): every triangle whose largest
    view-space edge ratio exceeds ``threshold`` splits that edge (the first
    of equal ones); then, while the triangle count after the splits exceeds
    ``budget`` (negative: no budget), the triangle with the lowest coverage
    (lowest index among equal counts) is removed (a triangle that would have
    split removes two).  Returns the plan: per output triangle, parent << 3 |
    op (op 0 copy, 1 + 2e + c child c of edge e), survivors in index order,
    the two children of a split in place of their parent."""
    ratios = np.asarray(ratios, np.float32)
    thr = np.float32(threshold)
    T = len(counts)
    split = []
    for t in range(T):
        e = 0
        for k in (1, 2):
            if ratios[t, k] > ratios[t, e]:
                e = k
        split.append(e if ratios[t, e] > thr else -1)
    n = T + sum(1 for e in split if e >= 0)
    removed = set()
    if budget >= 0:
        for t in sorted(range(T), key=lambda u: (int(counts[u]), u)):
            if n <= budget:
                break
            removed.add(t)
            n -= 2 if split[t] >= 0 else 1
    plan = []
    for t in range(T):
        if t in removed:
            continue
        if split[t] < 0:
            plan.append(t << 3)
        else:
            plan += [(t << 3) | (1 + 2 * split[t]), (t << 3) | (2 + 2 * split[t])]
    return np.array(plan, np.int32)


def adapt_plan_fill(counts, ratios, target: int):
    """The random-initialisation procedure (supplementary "Random Triangle
    Soup Initialization") as one round: triangles with no coverage in any
    training image are removed; then, while fewer than ``target`` remain,
    the survivors with the longest edges (largest ratio; lower index first
    among equal ones) split that edge, each at most once per round.  Plan
    codes as adapt_plan."""
    ratios = np.asarray(ratios, np.float32)
    T = len(counts)
    keep = [t for t in range(T) if int(counts[t]) > 0]
    longest = {}
    for t in keep:
        e = 0
        for k in (1, 2):
            if ratios[t, k] > ratios[t, e]:
                e = k
        longest[t] = e
    n_split = max(0, min(int(target) - len(keep), len(keep)))
    order = sorted(keep, key=lambda t: (-float(ratios[t, longest[t]]), t))
    split = set(order[:n_split])
    plan = []
    for t in keep:
        if t in split:
            e = longest[t]
            plan += [(t << 3) | (1 + 2 * e), (t << 3) | (2 + 2 * e)]
        else:
            plan.append(t << 3)
    return np.array(plan, np.int32)


def soup_rebuild(verts, levels, r_min: int, r_max: int, plan):
    """(verts_out [n, 3, 3], levels_out) of a split/prune plan (or_soup_rebuild)."""
    v = _c(verts, np.float32)
    T = v.shape[0]
    C = levels[0].shape[2]
    flat = np.concatenate([_c(l, np.float32).reshape(-1) for l in levels])
    pl = _c(plan, np.int32)
    n = len(pl)
    vo = np.empty((n, 3, 3), np.float32)
    lo = np.empty(sum(n * level_V(R) * C for R in range(r_min, r_max + 1)), np.float32)
    lib().or_soup_rebuild(_p(v), _p(flat), T, r_min, r_max, C, _p(pl), n, _p(vo), _p(lo))
    parts, o = [], 0
    for R in range(r_min, r_max + 1):
        m = n * level_V(R) * C
        parts.append(lo[o:o + m].reshape(n, level_V(R), C))
        o += m
    return vo, parts


# ---------------------------------------------------------------- full passes
def forward(verts, tex, grid_n, cams, seeds, S=1, mode=MODE_STOCHASTIC, bg=None,
            order=None, rows=None, scan=False):
    """Brute-force forward.  Returns one dict per view with tri_id [S,H,W],
    bary [S,H,W,2], depth [S,H,W], n_front, n_cover [S,H,W], color [S,C-1,H,W].
    scan=True: the same results through object-order candidate lists (the
    bbox-scan timing mode)."""
    verts = _c(verts, np.float32); tex = _c(tex, np.float32)
    T, V, C = tex.shape
    cf, wh = _cams(cams)
    seeds = _c(seeds if seeds is not None else np.zeros(len(cams), np.uint64), np.uint64)
    bg = _c(bg if bg is not None else np.zeros(C - 1), np.float32)
    npx = sum(S * c.width * c.height for c in cams)
    tri = np.full(npx, -1, np.int32); bary = np.zeros(2 * npx, np.float32)
    depth = np.zeros(npx, np.float32); nf = np.zeros(npx, np.int32); nc = np.zeros(npx, np.int32)
    color = np.zeros(npx * (C - 1), np.float32)
    order_a = None if order is None else _c(order, np.int32)
    r0, r1 = (0, -1) if rows is None else rows
    rc = lib().or_forward(_p(verts), _p(tex), T, grid_n, C, _p(cf), _p(wh), _p(seeds), len(cams),
                          S, mode, _p(bg), _p(order_a), r0, r1,
                          _p(tri), _p(bary), _p(depth), _p(nf), _p(nc), _p(color), int(bool(scan)))
    assert rc == 0, rc
    out, o, oc = [], 0, 0
    for c in cams:
        n = S * c.height * c.width
        out.append(dict(
            tri_id=tri[o:o + n].reshape(S, c.height, c.width),
            bary=bary[2 * o:2 * (o + n)].reshape(S, c.height, c.width, 2),
            depth=depth[o:o + n].reshape(S, c.height, c.width),
            n_front=nf[o:o + n].reshape(S, c.height, c.width),
            n_cover=nc[o:o + n].reshape(S, c.height, c.width),
            color=color[oc:oc + n * (C - 1)].reshape(S, C - 1, c.height, c.width)))
        o += n; oc += n * (C - 1)
    return out


def backward(verts, tex, grid_n, cams, S, fwd, grad_color, score_w, flags=G_ALL, rows=None, scan=False):
    """Algorithm A1 step 2 plus vertex gradients, FP64 accumulation.
    fwd: list of per-view dicts (tri_id, bary, color); grad_color: list of
    [S,C-1,H,W]; score_w: list of [S,H,W].  Returns (grad_tex, grad_verts).
    scan=True: object-order candidate lists, identical results (timing mode)."""
    verts = _c(verts, np.float32); tex = _c(tex, np.float32)
    T, V, C = tex.shape
    cf, wh = _cams(cams)
    def cat(arrays, dt):   # one view: no copy
        return _c(arrays[0].reshape(-1) if len(arrays) == 1 else np.concatenate([a.ravel() for a in arrays]), dt)
    tri = cat([f["tri_id"] for f in fwd], np.int32)
    bary = cat([f["bary"] for f in fwd], np.float32)
    col = cat([f["color"] for f in fwd], np.float32)
    gc = cat(list(grad_color), np.float32)
    sw = cat(list(score_w), np.float32)
    gt = np.zeros(tex.shape, np.float64); gv = np.zeros(verts.shape, np.float64)
    r0, r1 = (0, -1) if rows is None else rows
    rc = lib().or_backward(_p(verts), _p(tex), T, grid_n, C, _p(cf), _p(wh), len(cams), S,
                           _p(tri), _p(bary), _p(col), _p(gc), _p(sw), flags, r0, r1, _p(gt), _p(gv),
                           int(bool(scan)))
    assert rc == 0, rc
    return gt, gv


def expected(verts, tex, grid_n, cams, targets, bg=None, with_grad=True):
    """Closed-form E[l] per view (l = squared error summed over channels and
    pixels) and its exact gradient w.r.t. the texture logits (FP64 logits)."""
    verts = _c(verts, np.float32); tex = _c(tex, np.float64)
    T, V, C = tex.shape
    cf, wh = _cams(cams)
    tg = _c(np.concatenate([t.ravel() for t in targets]), np.float32)
    bg = _c(bg if bg is not None else np.zeros(C - 1), np.float32)
    el = np.zeros(len(cams), np.float64)
    eg = np.zeros(tex.shape, np.float64) if with_grad else None
    rc = lib().or_expected(_p(verts), _p(tex), T, grid_n, C, _p(cf), _p(wh), len(cams),
                           _p(tg), _p(bg), _p(el), _p(eg))
    assert rc == 0, rc
    return el, eg
