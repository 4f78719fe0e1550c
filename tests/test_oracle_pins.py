"""Pins of the CPU oracle against what the paper and the mathematics fix.

These run without a GPU.  Each test names the property it pins; a plausible
mistake in the oracle (a dropped term, a wrong sign, index or fill rule, a
transposed operand) fails at least one of them.
"""
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from paper_2603_27151_gb300 import inputs as I
from tests import geom_ref as G


# ---------------------------------------------------------------- scalar math
def test_expf_within_two_ulp_of_exp(O):
    xs = np.concatenate([np.linspace(-87.0, 88.7, 120001), np.linspace(-1.0, 1.0, 20001),
                         [0.0, -0.0, 1e-30, -1e-30, 0.34657359, -0.34657359]]).astype(np.float32)
    worst = 0.0
    for x in xs:
        got = O.expf(float(x))
        ref = math.exp(float(x))
        ulp = float(np.spacing(np.float32(ref)))
        worst = max(worst, abs(got - ref) / ulp)
    assert worst <= 2.0, worst
    assert O.expf(0.0) == 1.0
    assert O.expf(89.0) == math.inf and O.expf(-104.0) == 0.0
    assert math.isnan(O.expf(float("nan")))
    # subnormal range: absolute error within two subnormal steps
    for x in np.linspace(-103.9, -87.4, 2001):
        assert abs(O.expf(float(x)) - math.exp(float(np.float32(x)))) <= 2 * 2.0 ** -149


def test_sigmoid_special_values_and_accuracy(O):
    assert O.sigmoidf(0.0) == 0.5
    assert O.sigmoidf(40.0) == 1.0          # opacity identically one
    assert O.sigmoidf(-1e4) == 0.0          # opacity identically zero
    for x in np.linspace(-20, 20, 4001).astype(np.float32):
        ref = 1.0 / (1.0 + math.exp(-float(x)))
        assert abs(O.sigmoidf(float(x)) - ref) <= 4 * float(np.spacing(np.float32(ref))), x


# ---------------------------------------------------------------- Philox
_TRITON_SCRIPT = textwrap.dedent("""
    import os, sys, json
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl
    @triton.jit
    def k(out_ptr, c_ptr, seed, n, BLOCK: tl.constexpr):
        i = tl.arange(0, BLOCK)
        m = i < n
        c0 = tl.load(c_ptr + 4 * i + 0, mask=m).to(tl.uint32, bitcast=True)
        c1 = tl.load(c_ptr + 4 * i + 1, mask=m).to(tl.uint32, bitcast=True)
        c2 = tl.load(c_ptr + 4 * i + 2, mask=m).to(tl.uint32, bitcast=True)
        c3 = tl.load(c_ptr + 4 * i + 3, mask=m).to(tl.uint32, bitcast=True)
        r0, r1, r2, r3 = tl.random.philox(seed, c0, c1, c2, c3)
        tl.store(out_ptr + 4 * i + 0, r0.to(tl.int32, bitcast=True), mask=m)
        tl.store(out_ptr + 4 * i + 1, r1.to(tl.int32, bitcast=True), mask=m)
        tl.store(out_ptr + 4 * i + 2, r2.to(tl.int32, bitcast=True), mask=m)
        tl.store(out_ptr + 4 * i + 3, r3.to(tl.int32, bitcast=True), mask=m)
    req = json.load(sys.stdin)
    res = []
    for seed, ctrs in req:
        c = torch.tensor(np.array(ctrs, np.uint32).view(np.int32).ravel())
        out = torch.zeros_like(c)
        k[(1,)](out, c, seed, len(ctrs), BLOCK=64)
        res.append(out.numpy().view(np.uint32).reshape(-1, 4).tolist())
    json.dump(res, sys.stdout)
""")


def test_philox_matches_an_independent_implementation(O):
    """Philox4x32-10 against Triton's implementation (run by its CPU
    interpreter): a different code base for the same published generator."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(123)
    req = []
    for seed in [0, 1, 0xFFFFFFFFFFFFFFFF, int(rng.integers(0, 2**63)), int(rng.integers(0, 2**63))]:
        ctrs = rng.integers(0, 2**32, (40, 4), dtype=np.uint64)
        ctrs[0] = 0
        ctrs[1] = 0xFFFFFFFF
        req.append([seed, ctrs.tolist()])
    import json
    p = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(req),
                       capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    res = json.loads(p.stdout)
    for (seed, ctrs), outs in zip(req, res):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for c, o in zip(ctrs, outs):
            assert O.philox(c, key).tolist() == o


def test_tau_is_uniform_on_the_2_24_grid(O):
    vals = np.array([O.tau(987654321, px, py, t, s)
                     for px in range(8) for py in range(8) for t in range(64) for s in range(8)])
    assert vals.min() >= 0.0 and vals.max() < 1.0
    assert np.all(vals * 2.0 ** 24 == np.round(vals * 2.0 ** 24))
    h, _ = np.histogram(vals, bins=64, range=(0, 1))
    e = len(vals) / 64.0
    chi2 = ((h - e) ** 2 / e).sum()
    assert chi2 < 120, chi2          # 63 dof; p ~ 1e-5 bound
    # the four words of one block serve samples 4k..4k+3; other counters differ
    assert O.tau(5, 1, 2, 3, 0) != O.tau(5, 1, 2, 3, 4)
    assert O.tau(5, 1, 2, 3, 0) != O.tau(6, 1, 2, 3, 0)


# ---------------------------------------------------------------- texture decode
def test_texel_count_matches_the_paper(O):
    """R_max = 5 gives (2^4+1)(2^5+1) = 561 feature vertices (supplementary
    "Data Size"), and 4096^2 / 561 ~ 29,905 triangles fit a 4K atlas."""
    N = 32
    assert I.n_texels(N) == (2 ** 4 + 1) * (2 ** 5 + 1) == 561
    assert 4096 ** 2 // 561 == 29905
    used = set()
    for b1 in np.linspace(0, 1, 161):
        for b2 in np.linspace(0, 1, 161):
            if b1 + b2 <= 1.0:
                idx, _ = O.cell(N, b1, b2)
                used.update(idx.tolist())
    assert used == set(range(561))


@pytest.mark.parametrize("N", [1, 2, 4, 8, 32])
def test_lookup_reproduces_linear_functions(O, N):
    rng = np.random.default_rng(N)
    c = rng.standard_normal(3)
    tab = G.grid_index_table(N)
    grid = np.zeros(len(tab), np.float32)
    for (i, j), k in tab.items():
        grid[k] = c[0] + c[1] * i / N + c[2] * j / N
    for _ in range(400):
        b = rng.dirichlet([1, 1, 1])
        got = O.lookup(grid, N, b[1], b[2])
        assert abs(got - (c[0] + c[1] * np.float32(b[1]) + c[2] * np.float32(b[2]))) < 2e-5
    const = np.full(len(tab), 0.3125, np.float32)
    for _ in range(100):
        b = rng.dirichlet([1, 1, 1])
        assert O.lookup(const, N, b[1], b[2]) == np.float32(0.3125)
    # grid vertices return their own value
    rnd = rng.standard_normal(len(tab)).astype(np.float32)
    for (i, j), k in tab.items():
        assert abs(O.lookup(rnd, N, i / N, j / N) - rnd[k]) < 1e-6


def test_lookup_is_continuous_across_micro_triangles(O):
    """Piecewise-linear interpolation over the subdivided triangle is
    continuous: no jumps along lines that cross many micro-triangle edges."""
    N = 8
    rng = np.random.default_rng(7)
    grid = rng.standard_normal(I.n_texels(N)).astype(np.float32)
    for _ in range(20):
        p0, p1 = rng.dirichlet([1, 1, 1]), rng.dirichlet([1, 1, 1])
        ts = np.linspace(0, 1, 4001)
        vals = np.array([O.lookup(grid, N, *(p0 + t * (p1 - p0))[1:]) for t in ts])
        step = np.abs(np.diff(vals)).max()
        assert step < 4 * N * np.abs(grid).max() * 2.0 / 4000 + 1e-5, step


# ---------------------------------------------------------------- coverage, depth
def _plane_mesh(n, lo, hi, rng, jitter=True):
    """Regular grid of (n+1)^2 points in the plane z = 0 split into 2n^2
    triangles with random diagonals; shared edges use identical vertices."""
    xs = np.linspace(lo, hi, n + 1)
    P = np.zeros((n + 1, n + 1, 3), np.float32)
    for a in range(n + 1):
        for b in range(n + 1):
            P[a, b] = (xs[a], xs[b], 0.0)
            if jitter and 0 < a < n and 0 < b < n:
                P[a, b, :2] += rng.uniform(-0.3, 0.3, 2) * (hi - lo) / n
    tris = []
    for a in range(n):
        for b in range(n):
            q = [P[a, b], P[a + 1, b], P[a + 1, b + 1], P[a, b + 1]]
            if rng.random() < 0.5:
                tris += [[q[0], q[1], q[2]], [q[0], q[2], q[3]]]
            else:
                tris += [[q[0], q[1], q[3]], [q[1], q[2], q[3]]]
    return np.array(tris, np.float32)


@pytest.mark.parametrize("jitter", [False, True])
def test_shared_edges_cover_every_pixel_exactly_once(O, jitter):
    """Top-left fill rule: a tiling covers each pixel centre once, including
    centres that lie exactly on shared edges and vertices (the unjittered grid
    puts edges and vertices on pixel centres: screen x = 4 world x + 24)."""
    rng = np.random.default_rng(11 + jitter)
    cam = G.manual_camera(48, 48, 16.0, 4.0)
    verts = _plane_mesh(8, -4.875, 3.125, rng, jitter)     # grid step 1.0 world = 4 px, offset 0.5 px
    T = len(verts)
    tex = np.full((T, 3, 2), -1e4, np.float32)               # alpha == 0: count covered fragments only
    out = O.forward(verts, tex, 1, [cam], np.zeros(1, np.uint64))[0]
    nc = out["n_cover"][0]
    assert nc.max() == 1
    # every centre strictly inside the outer square [-4.875, 3.125]^2 is covered
    wx = (np.arange(48) + 0.5 - 24) / 4.0          # world x of each pixel column
    wy = (24 - (np.arange(48) + 0.5)) / 4.0        # world y of each pixel row (screen y is down)
    in_x = (wx > -4.875 + 1e-3) & (wx < 3.125 - 1e-3)
    in_y = (wy > -4.875 + 1e-3) & (wy < 3.125 - 1e-3)
    assert np.all(nc[np.ix_(in_y, in_x)] == 1)
    # the outer boundary runs through pixel centres: the fill rule keeps the
    # left and top sides and drops the right and bottom ones, so the count is
    # exactly the area in pixels (8 world units = 32 px per side)
    assert nc.sum() == 32 * 32
    # screen x in [4.5, 36.5], screen y in [11.5, 43.5]: the left column (4)
    # and top row (11) are owned, the right column (36) and bottom row (43) not
    assert np.all(nc[12:43, 4] == 1) and np.all(nc[12:43, 36] == 0)
    assert np.all(nc[11, 5:36] == 1) and np.all(nc[43, 5:36] == 0)
    assert np.all(out["tri_id"][0] == -1) and np.all(out["n_front"][0] == nc)


def test_depth_and_barycentrics_match_ray_plane_intersection(O):
    sc = I.plain_small()
    cam = sc.cams[0]
    rng = np.random.default_rng(3)
    checked = 0
    for t in range(sc.T):
        Vc = np.stack([G.to_cam(cam, p) for p in sc.verts[t]])
        P = np.stack([G.project(cam, v) for v in Vc])
        lo = np.clip(np.floor(P.min(0)), 0, 63).astype(int)
        hi = np.clip(np.ceil(P.max(0)), 1, 64).astype(int)
        for _ in range(30):
            px, py = int(rng.integers(lo[0], hi[0])), int(rng.integers(lo[1], hi[1]))
            cov, rho, D, b1, b2 = O.fragment(sc.verts[t], cam, px, py)
            dist = G.edge_dist(P, (px + 0.5, py + 0.5))
            if dist.min() > 0.01:
                assert cov
            if dist.min() < -0.01:
                assert not cov
            if cov and dist.min() > 0.05:
                b0r, b1r, b2r, z = G.ray_hit(cam, Vc, px + 0.5, py + 0.5)
                scale = max(1.0, 1.0 / max(1e-3, abs(np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0]])) / 2) ** 0.5))
                assert abs(D - z) <= 2e-3 * z
                assert abs(rho - 1.0 / z) <= 2e-3 / z
                assert abs(b1 - b1r) < 5e-3 * scale and abs(b2 - b2r) < 5e-3 * scale
                checked += 1
    assert checked > 200


def _zbuffer_reference(verts, cam):
    """Textbook z-buffer in FP64 on the continuous triangles; returns the
    winner per pixel and a mask of pixels whose answer is unambiguous."""
    W, H = cam.width, cam.height
    win = np.full((H, W), -1)
    ok = np.ones((H, W), bool)
    Vcs = [np.stack([G.to_cam(cam, p) for p in tri]) for tri in verts]
    Ps = [np.stack([G.project(cam, v) for v in Vc]) for Vc in Vcs]
    for py in range(H):
        for px in range(W):
            x = (px + 0.5, py + 0.5)
            cands, amb = [], False
            for t, (Vc, P) in enumerate(zip(Vcs, Ps)):
                d = G.edge_dist(P, x).min()
                if abs(d) < 0.02:
                    amb = True
                if d > 0:
                    cands.append((G.ray_hit(cam, Vc, *x)[3], t))
            cands.sort()
            if len(cands) >= 2 and cands[1][0] - cands[0][0] < 1e-4 * cands[0][0]:
                amb = True
            win[py, px] = cands[0][1] if cands else -1
            ok[py, px] = not amb
    return win, ok


def test_opacity_one_reduces_to_a_plain_zbuffer(O):
    """Eq. 2 special case: alpha == 1 selects the foremost fragment."""
    sc = I.plain_small()
    tex = sc.tex.copy()
    tex[..., -1] = 40.0
    out = O.forward(sc.verts, tex, sc.grid_n, sc.cams, sc.seeds)[0]
    ref, ok = _zbuffer_reference(sc.verts, sc.cams[0])
    assert ok.mean() > 0.85
    assert np.array_equal(out["tri_id"][0][ok], ref[ok])
    assert np.all(out["n_front"][0] == 0)


def test_opacity_zero_gives_the_background(O):
    sc = I.plain_small()
    tex = sc.tex.copy()
    tex[..., -1] = -1e4
    bg = np.array([0.1, 0.2, 0.3], np.float32)
    out = O.forward(sc.verts, tex, sc.grid_n, sc.cams, sc.seeds, bg=bg)[0]
    assert np.all(out["tri_id"] == -1)
    assert np.array_equal(out["n_front"], out["n_cover"]) and out["n_cover"].sum() > 1000
    assert np.all(out["color"][0] == bg[:, None, None])


def test_threshold_half_is_binary_opacity_selection(O):
    """Eq. 3: the foremost fragment with alpha(b) > 0.5."""
    sc = I.plain_small()
    out = O.forward(sc.verts, sc.tex, sc.grid_n, sc.cams, sc.seeds, mode=O.MODE_THRESHOLD_HALF)[0]
    act = O.activate(sc.tex)
    cam = sc.cams[0]
    for py in range(0, 64, 3):
        for px in range(0, 64, 3):
            best = (-1, 0.0)
            for t in range(sc.T):
                cov, rho, D, b1, b2 = O.fragment(sc.verts[t], cam, px, py)
                if cov and O.lookup(act[t, :, -1], sc.grid_n, b1, b2) > 0.5:
                    if best[0] < 0 or rho > best[1]:
                        best = (t, rho)
            assert out["tri_id"][0, py, px] == best[0]


def test_selection_is_independent_of_triangle_order(O):
    """The z-buffer arg-min of Eq. 5 needs no sorting: visiting triangles in
    any order gives identical buffers."""
    sc = I.plain_small()
    a = O.forward(sc.verts, sc.tex, sc.grid_n, sc.cams, sc.seeds, S=2)[0]
    for seed in range(3):
        order = np.random.default_rng(seed).permutation(sc.T)
        b = O.forward(sc.verts, sc.tex, sc.grid_n, sc.cams, sc.seeds, S=2, order=order)[0]
        for k in a:
            assert np.array_equal(a[k], b[k]), k


def _flat_tri(z, half):
    return np.array([[-half, -half, z], [half, -half * 0.9, z], [0.1 * half, half, z]], np.float32)


def test_monte_carlo_coverage_converges_to_opacity(O):
    cam = G.manual_camera(16, 16, 16.0, 4.0)
    verts = _flat_tri(0.0, 6.0)[None]
    theta = 0.4
    tex = np.full((1, 3, 2), theta, np.float32)
    S = 512
    out = O.forward(verts, tex, 1, [cam], np.array([42], np.uint64), S=S)[0]
    cov = out["n_cover"] > 0
    hit = (out["tri_id"] == 0)[cov]
    a = 1.0 / (1.0 + math.exp(-theta))
    n = hit.size
    assert n > 50000
    assert abs(hit.mean() - a) < 5 * math.sqrt(a * (1 - a) / n)


def test_two_layers_follow_the_transmittance_weights(O):
    """Eq. 6 / A1: P(front) = a1, P(back) = (1-a1) a2, P(none) = (1-a1)(1-a2)."""
    cam = G.manual_camera(16, 16, 16.0, 4.0)
    verts = np.stack([_flat_tri(-0.5, 6.0), _flat_tri(0.5, 6.0)])   # index 1 is in front (z = 0.5 is nearer)
    th = np.array([0.7, -0.3], np.float32)
    tex = np.zeros((2, 3, 2), np.float32)
    tex[0, :, -1], tex[1, :, -1] = th[0], th[1]
    S = 512
    out = O.forward(verts, tex, 1, [cam], np.array([7], np.uint64), S=S)[0]
    both = out["n_cover"] == 2
    w = out["tri_id"][both]
    a_back, a_front = 1 / (1 + np.exp(-th.astype(np.float64)))
    p = np.array([a_front, (1 - a_front) * a_back, (1 - a_front) * (1 - a_back)])
    cnt = np.array([(w == 1).sum(), (w == 0).sum(), (w == -1).sum()])
    e = p * cnt.sum()
    chi2 = ((cnt - e) ** 2 / e).sum()
    assert cnt.sum() > 50000 and chi2 < 20, (cnt, e)


# ---------------------------------------------------------------- gradients
def _small_scene(seed=0, T=10, N=2, C=3, W=20, H=18):
    rng = np.random.default_rng(seed)
    verts = I.box_soup(T, 1.2, rng, half=0.6)
    tex = I.logits(T, N, C, rng)
    cam = I.look_at(I.sphere_eyes(1, 3.0, rng)[0], W, H)
    target = rng.uniform(0, 1, (C - 1, H, W)).astype(np.float32)
    return verts, tex, cam, target


def test_expected_gradient_equals_finite_differences_of_expected_loss(O):
    """Eq. 7-9 and Algorithm A1 together: the closed-form expectation of the
    estimator equals the derivative of E[l] (FP64 central differences)."""
    verts, tex, cam, target = _small_scene()
    t64 = tex.astype(np.float64)
    L, g = O.expected(verts, t64, 2, [cam], [target])
    assert L[0] > 0
    rng = np.random.default_rng(1)
    nz = np.argwhere(np.abs(g) > 1e-4 * np.abs(g).max())
    opa = nz[nz[:, 2] == tex.shape[2] - 1]
    col = nz[nz[:, 2] < tex.shape[2] - 1]
    pick = np.concatenate([opa[rng.choice(len(opa), 25, replace=False)],
                           col[rng.choice(len(col), 15, replace=False)]])
    h = 1e-5
    for (t, k, c) in pick:
        tp, tm = t64.copy(), t64.copy()
        tp[t, k, c] += h
        tm[t, k, c] -= h
        fd = (O.expected(verts, tp, 2, [cam], [target], with_grad=False)[0][0]
              - O.expected(verts, tm, 2, [cam], [target], with_grad=False)[0][0]) / (2 * h)
        assert abs(fd - g[t, k, c]) <= 1e-6 * max(abs(g[t, k, c]), 1e-3 * np.abs(g).max()), (t, k, c, fd, g[t, k, c])


def test_sampled_estimator_averages_to_the_expected_gradient(O):
    """The oracle's Algorithm-A1 backward, averaged over masks, is unbiased."""
    verts, tex, cam, target = _small_scene()
    _, eg = O.expected(verts, tex.astype(np.float64), 2, [cam], [target])
    S = 256
    ests = []
    for rep in range(8):
        f = O.forward(verts, tex, 2, [cam], np.array([1000 + rep], np.uint64), S=S)[0]
        diff = f["color"] - target[None]
        ell = (diff.astype(np.float64) ** 2).sum(1)
        gcol = (2.0 * diff / S).astype(np.float32)
        sw = (ell / S).astype(np.float32)
        gt, _ = O.backward(verts, tex, 2, [cam], S, [f], [gcol], [sw], flags=O.G_TEX | O.G_SCORE)
        ests.append(gt)
    ests = np.array(ests)
    m, se = ests.mean(0), ests.std(0, ddof=1) / math.sqrt(len(ests))
    big = np.abs(eg) > 0.05 * np.abs(eg).max()
    z = np.abs(m - eg)[big] / (se[big] + 1e-12)
    assert big.sum() > 20
    assert np.mean(z < 4) > 0.97 and z.max() < 7, z.max()
    rel = np.linalg.norm(m - eg) / np.linalg.norm(eg)
    assert rel < 0.08, rel


def _decode64(th, N, idx, wa, wb):
    a = 1.0 / (1.0 + np.exp(-th))
    return a[idx[0]] + wa * (a[idx[1]] - a[idx[0]]) + wb * (a[idx[2]] - a[idx[0]])


def test_colour_gradient_equals_finite_differences(O):
    """Algorithm A1 2(a): colour gradient through the decode and the sigmoid."""
    verts, tex, cam, _ = _small_scene(seed=3, C=4)
    tex[..., -1] = 40.0                       # fixed visibility
    f = O.forward(verts, tex, 2, [cam], np.zeros(1, np.uint64))[0]
    rng = np.random.default_rng(0)
    Gc = rng.standard_normal(f["color"].shape).astype(np.float32)
    gt, _ = O.backward(verts, tex, 2, [cam], 1, [f], [Gc], [np.zeros((1, 18, 20), np.float32)],
                       flags=O.G_TEX)
    cells = {}
    for py in range(18):
        for px in range(20):
            t = f["tri_id"][0, py, px]
            if t >= 0:
                cells[(py, px)] = (t, *O.cell(2, *f["bary"][0, py, px]))

    def loss(th):
        L = 0.0
        for (py, px), (t, idx, w) in cells.items():
            for c in range(3):
                L += Gc[0, c, py, px] * _decode64(th[t, :, c], 2, idx, float(w[0]), float(w[1]))
        return L

    th = tex.astype(np.float64)
    nz = np.argwhere(np.abs(gt) > 1e-6)
    assert len(nz) > 30
    for (t, k, c) in nz[rng.choice(len(nz), 20, replace=False)]:
        tp, tm = th.copy(), th.copy()
        tp[t, k, c] += 1e-6
        tm[t, k, c] -= 1e-6
        fd = (loss(tp) - loss(tm)) / 2e-6
        assert abs(fd - gt[t, k, c]) < 1e-6 * max(1.0, abs(fd)), (fd, gt[t, k, c])


def test_interior_vertex_gradient_equals_finite_differences(O):
    """First term of Eq. 8 for the vertices: colour moves with the
    perspective-correct barycentrics of the selected fragment."""
    verts, tex, cam, _ = _small_scene(seed=5, C=4, N=4)
    tex[..., -1] = 40.0
    N = 4
    f = O.forward(verts, tex, N, [cam], np.zeros(1, np.uint64))[0]
    rng = np.random.default_rng(2)
    Gc = rng.standard_normal(f["color"].shape).astype(np.float32)
    _, gv = O.backward(verts, tex, N, [cam], 1, [f], [Gc], [np.zeros((1, 18, 20), np.float32)],
                       flags=O.G_INTERIOR)
    act = 1.0 / (1.0 + np.exp(-tex.astype(np.float64)))
    tab = G.grid_index_table(N)
    pix = []
    for py in range(18):
        for px in range(20):
            t = f["tri_id"][0, py, px]
            if t < 0:
                continue
            b1, b2 = (float(x) for x in f["bary"][0, py, px])
            u, v = N * np.float32(b1), N * np.float32(b2)
            i = min(max(int(np.floor(u)), 0), N - 1)
            j = min(max(int(np.floor(v)), 0), N - 1 - i)
            lower = (u - i) + (v - j) <= 1.0 or i + j == N - 1
            pix.append((py, px, t, i, j, lower))

    def loss(vv):
        L = 0.0
        for (py, px, t, i, j, lower) in pix:
            Vc = np.stack([G.to_cam(cam, p) for p in vv[t]])
            _, b1, b2, _ = G.ray_hit(cam, Vc, px + 0.5, py + 0.5)
            fu, fv = N * b1 - i, N * b2 - j
            if lower:
                k0, k1, k2, wa, wb = tab[(i, j)], tab[(i + 1, j)], tab[(i, j + 1)], fu, fv
            else:
                k0, k1, k2, wa, wb = tab[(i + 1, j + 1)], tab[(i, j + 1)], tab[(i + 1, j)], 1 - fu, 1 - fv
            for c in range(3):
                a = act[t, :, c]
                L += Gc[0, c, py, px] * (a[k0] + wa * (a[k1] - a[k0]) + wb * (a[k2] - a[k0]))
        return L

    vv = verts.astype(np.float64)
    ts = np.unique([p[2] for p in pix])
    assert len(ts) >= 3
    for t in ts[:4]:
        for m in range(3):
            for ax in range(3):
                vp, vm = vv.copy(), vv.copy()
                vp[t, m, ax] += 1e-6
                vm[t, m, ax] -= 1e-6
                fd = (loss(vp) - loss(vm)) / 2e-6
                assert abs(fd - gv[t, m, ax]) < 1e-4 * max(abs(fd), 1e-2 * np.abs(gv).max()), (t, m, ax, fd, gv[t, m, ax])


@pytest.mark.parametrize("verts", [
    [[-5.1, -4.3, 0.6], [6.2, -3.1, -0.8], [-0.7, 5.9, 0.3]],      # generic edge directions
    [[-0.3, -30.0, 0.4], [0.5, 30.0, -0.5], [-30.0, 0.5, 0.1]],    # one edge, 0.8 degrees from vertical, in view
])
def test_silhouette_gradient_matches_antialiased_finite_differences(O, verts):
    """Edge gradients (Sec. 3.2, after rasterized edge gradients): for one
    opaque triangle over the background, the pair-wise boundary term
    approximates the derivative of the box-filtered (area-coverage) loss.
    A point-sampled image cannot see where inside a pixel an edge lies, so the
    two agree on average over sub-pixel placements: both sides are summed over
    16 sub-pixel shifts of the principal point on a rank-1 lattice (stratified
    in x and in y)."""
    W = H = 40
    verts = np.array([verts], np.float32)
    C = 4
    tex = np.full((1, 3, C), 0.8, np.float32)
    tex[..., -1] = 40.0
    col = 1.0 / (1.0 + math.exp(-0.8))
    yy, xx = np.mgrid[0:H, 0:W]
    target = np.stack([0.02 + 0.002 * xx, 0.1 - 0.002 * yy, 0.05 + 0.001 * (xx + yy)]).astype(np.float64)
    g_sum, fd_sum = np.zeros(9), np.zeros(9)
    norms = []
    for k in range(16):
        cam = G.manual_camera(W, H, 10.0, 4.0)
        cam.cx += (k + 0.37) / 16.0
        cam.cy += ((7 * k) % 16 + 0.61) / 16.0
        f = O.forward(verts, tex, 1, [cam], np.zeros(1, np.uint64))[0]
        gcol = (2.0 * (f["color"][0] - target))[None].astype(np.float32)
        _, gv = O.backward(verts, tex, 1, [cam], 1, [f], [gcol], [np.zeros((1, H, W), np.float32)],
                           flags=O.G_EDGE)
        g_sum += gv.reshape(-1)
        norms.append(np.linalg.norm(gv))
        P0 = np.stack([G.project(cam, G.to_cam(cam, p)) for p in verts[0].astype(np.float64)])
        near = [(py, px) for py in range(H) for px in range(W)
                if np.abs(G.edge_dist(P0, (px + 0.5, py + 0.5))).min() < 1.5]

        def aa_loss(vv):
            P = np.stack([G.project(cam, G.to_cam(cam, p)) for p in vv[0]])
            L = 0.0
            for (py, px) in near:        # pixels away from every edge do not change
                a = G.clip_area(P, px, py, px + 1, py + 1)
                L += ((col * a - target[:, py, px]) ** 2).sum()
            return L

        vv = verts.astype(np.float64)
        for q in range(9):
            vp, vm = vv.copy(), vv.copy()
            vp.reshape(-1)[q] += 1e-5
            vm.reshape(-1)[q] -= 1e-5
            fd_sum[q] += (aa_loss(vp) - aa_loss(vm)) / 2e-5
    cos = g_sum @ fd_sum / (np.linalg.norm(g_sum) * np.linalg.norm(fd_sum))
    ratio = np.linalg.norm(g_sum) / np.linalg.norm(fd_sum)
    # measured: cos 0.99999 and ratios 1.004 / 1.002 for the two cases, so
    # the absolute weight of the silhouette term is pinned to about 1%
    assert cos > 0.9995, (cos, g_sum, fd_sum)
    assert abs(ratio - 1.0) < 0.015, (ratio, g_sum, fd_sum)
    # weighting each pair axis by the squared normal component keeps every
    # crossing's contribution bounded: the estimate barely moves with the
    # sub-pixel placement (weighting the other axis is also unbiased on
    # average but jumps between 0 and ~70x for a near-axis-aligned edge)
    norms = np.array(norms)
    assert norms.std() / norms.mean() < 0.25, norms


def test_implicit_boundary_gradient_has_zero_mean_under_translation(O):
    """A uniform-opacity, uniform-colour triangle that covers the whole image:
    translating it in its plane leaves the image distribution unchanged, so
    the mask-boundary gradient has zero mean over masks."""
    W = H = 16
    cam = G.manual_camera(W, H, 16.0, 4.0)
    verts = _flat_tri(0.0, 8.0)[None]
    tex = np.zeros((1, 3, 4), np.float32)
    tex[..., :3] = 1.0
    tex[..., -1] = 0.0
    target = np.full((3, H, W), 0.25)
    S = 64
    vals = []
    for rep in range(24):
        f = O.forward(verts, tex, 1, [cam], np.array([500 + rep], np.uint64), S=S)[0]
        gcol = (2.0 * (f["color"] - target[None]) / S).astype(np.float32)
        _, gv = O.backward(verts, tex, 1, [cam], S, [f], [gcol], [np.zeros((S, H, W), np.float32)],
                           flags=O.G_EDGE)
        vals.append(gv.sum(axis=1)[0, :2])       # in-plane translation
    vals = np.array(vals)
    m, se = vals.mean(0), vals.std(0, ddof=1) / math.sqrt(len(vals))
    assert np.all(np.abs(vals).max(0) > 0)       # the term is active
    assert np.all(np.abs(m) < 5 * se), (m, se)


def test_implicit_boundary_gradient_is_unbiased_for_a_moving_opacity_field(O):
    """Mask-induced (implicit) boundaries: a triangle covering the whole image
    with an opacity that varies linearly over it.  Moving a vertex moves the
    opacity field with the surface, so E[l] = sum_p alpha_p l(c) +
    (1 - alpha_p) l(bg) changes; averaged over masks, the implicit edge term
    must equal the derivative of that expectation (central differences on the
    continuous barycentrics).  Pairs only exist inside the image, so the
    estimator sees (W-1)/W of the pixel steps of a linear field."""
    W = H = 48
    cam = G.manual_camera(W, H, 24.0, 4.0)
    verts = np.array([[[-14.0, -12.0, 0.5], [19.0, -11.0, -0.6], [-2.5, 19.0, 0.2]]], np.float32)
    al = np.array([0.15, 0.85, 0.5])
    tex = np.zeros((1, 3, 4), np.float32)
    tex[0, :, -1] = np.log(al / (1 - al))
    tex[0, :, :3] = 1.0
    N = 1
    a32 = O.activate(tex)[0, :, -1].astype(np.float64)
    c = 1.0 / (1.0 + math.exp(-1.0))
    tgt = 0.25
    l_c, l_bg = 3 * (c - tgt) ** 2, 3 * tgt ** 2

    def e_loss(vv):
        Vc = np.stack([G.to_cam(cam, p) for p in vv[0]])
        L = 0.0
        for py in range(H):
            for px in range(W):
                b0, b1, b2, _ = G.ray_hit(cam, Vc, px + 0.5, py + 0.5)
                a = b0 * a32[0] + b1 * a32[1] + b2 * a32[2]
                L += a * l_c + (1 - a) * l_bg
        return L

    vv = verts.astype(np.float64)
    fd = np.zeros(9)
    for q in range(9):
        vp, vm = vv.copy(), vv.copy()
        vp.reshape(-1)[q] += 1e-4
        vm.reshape(-1)[q] -= 1e-4
        fd[q] = (e_loss(vp) - e_loss(vm)) / 2e-4
    S = 64
    acc = []
    for rep in range(16):
        f = O.forward(verts, tex, N, [cam], np.array([900 + rep], np.uint64), S=S)[0]
        assert np.all(f["n_cover"] == 1)                 # no silhouette anywhere
        gcol = (2.0 * (f["color"] - tgt) / S).astype(np.float32)
        _, gv = O.backward(verts, tex, N, [cam], S, [f], [gcol], [np.zeros((S, H, W), np.float32)],
                           flags=O.G_EDGE)
        acc.append(gv.reshape(-1))
    g = np.mean(acc, 0)
    cos = g @ fd / (np.linalg.norm(g) * np.linalg.norm(fd))
    ratio = np.linalg.norm(g) / np.linalg.norm(fd)
    assert cos > 0.995, (cos, g, fd)
    assert abs(ratio - (W - 1) / W) < 0.025, (ratio, g, fd)
    # unbiasedness component by component: each mean within 4 standard
    # errors of the expected derivative (measured: |z| <= 1.7)
    se = np.std(acc, 0, ddof=1) / math.sqrt(len(acc))
    z = (g - fd * (W - 1) / W) / se
    assert np.all(np.abs(z) < 4.0), z
