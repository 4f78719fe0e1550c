"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs.  Visibility (triangle id, n_front, barycentrics, depth)
must match bit for bit; colours within 1e-5 relative; gradients within 1e-4
relative of the oracle's identical estimator (|g - ref| <= 1e-4 max(|ref|,
1e-3 max|ref|), FP32 atomics against FP64 sums)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2603_27151_gb300 import inputs as I
from tests import geom_ref as G
from tests.gpu_helpers import assert_forward_equal, gpu_backward, gpu_forward, grad_mismatch, upstream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_27151_gb300 import native as N
    c = N.Context(0)
    yield c
    c.close()


def _oracle_fwd(sc, S=None, mode=0):
    return O.forward(sc.verts, sc.tex, sc.grid_n, sc.cams, sc.seeds, S=S or sc.samples, mode=mode, bg=sc.bg)


# ------------------------------------------------------------------ forward
def test_forward_plain_small(ctx):
    sc = I.plain_small()
    _, got, _ = gpu_forward(ctx, sc)
    assert_forward_equal(got, _oracle_fwd(sc))


@pytest.mark.parametrize("S", [2, 4, 5, 9])
def test_forward_sample_groups(ctx, S):
    """Samples share one Philox block per group of four; ragged last groups."""
    sc = I.plain_small(soup_seed=3, mask_seed=4)
    _, got, _ = gpu_forward(ctx, sc, S=S)
    assert_forward_equal(got, _oracle_fwd(sc, S=S))


def test_forward_threshold_half(ctx):
    sc = I.plain_small(soup_seed=5)
    _, got, _ = gpu_forward(ctx, sc, mode=1)
    assert_forward_equal(got, _oracle_fwd(sc, mode=1))


def test_forward_batched_views_mixed_resolutions(ctx):
    """2,000 triangles, 8 views at 128^2 / 256^2 / 320x240 in one launch."""
    sc = I.batched_views()
    _, got, _ = gpu_forward(ctx, sc)
    assert_forward_equal(got, _oracle_fwd(sc))


def _edge_scene():
    """Ragged image sizes, a 1x1 view, a view looking away from the soup,
    triangles crossing the camera plane, degenerate and huge triangles."""
    rng = np.random.default_rng(21)
    verts = I.box_soup(300, 0.3, rng)
    verts[0] = [[0, 0, 0], [0.5, 0.5, 0.5], [1.0, 1.0, 1.0]]          # collinear: zero area
    verts[1] = [[0.2, 0.2, 0.2]] * 3                                     # a point
    verts[2] = [[-9.0, -9.0, 0.1], [9.0, -9.0, 0.0], [0.0, 9.0, -0.1]]   # huge: covers many tiles
    verts[3] = [[0.0, 0.0, 2.5], [0.3, 0.0, 3.5], [0.0, 0.3, 2.8]]       # near the first camera
    tex = I.logits(300, 3, 5, rng)
    cams = [I.look_at([0.0, 0.0, 3.0], 37, 23), I.look_at([2.0, 1.0, 2.0], 1, 1),
            I.look_at([0.0, 3.0, 0.0], 48, 33)]
    away = I.look_at([0.0, 0.0, 3.0], 20, 20)
    away.R = (-away.R.astype(np.float64)).astype(np.float32)   # looks away from the soup
    away.t = np.array([0.0, 0.0, -10.0], np.float32)
    cams.append(away)
    return I.Scene(verts, tex, 3, cams, I.mask_seeds(77, 4), 1, np.array([0.1, 0.2, 0.3, 0.4], np.float32))


def test_forward_edge_cases(ctx):
    sc = _edge_scene()
    _, got, _ = gpu_forward(ctx, sc, S=3)
    ref = _oracle_fwd(sc, S=3)
    assert_forward_equal(got, ref)
    assert np.all(ref[3]["tri_id"] == -1)


def test_forward_exact_tiling_on_pixel_centres(ctx):
    """Shared edges through pixel centres: each centre covered once (fill rule)."""
    from tests.test_oracle_pins import _plane_mesh
    rng = np.random.default_rng(11)
    cam = G.manual_camera(48, 48, 16.0, 4.0)
    verts = _plane_mesh(8, -4.875, 3.125, rng, False)
    tex = np.full((len(verts), 3, 2), -1e4, np.float32)
    sc = I.Scene(verts, tex, 1, [cam], I.mask_seeds(1, 1), 1, np.zeros(1, np.float32))
    _, got, _ = gpu_forward(ctx, sc)
    ref = _oracle_fwd(sc)
    assert_forward_equal(got, ref)
    assert got[0]["n_front"].sum() == 32 * 32


def test_fragment_count_matches_oracle(ctx):
    sc = I.batched_views()
    import torch
    sid = ctx.soup_upload(torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.tex).cuda(), sc.grid_n)
    n = ctx.fragment_count(sid, sc.cams)
    ref = _oracle_fwd(sc)
    assert n == sum(int(f["n_cover"].sum()) for f in ref)


# ------------------------------------------------------------------ backward
def _check_grads(gt, gv, rt, rv, what):
    for got, want, name in ((gt, rt, "grad_tex"), (gv, rv, "grad_verts")):
        if not np.any(want):
            assert not np.any(got), "%s %s should be zero" % (what, name)
            continue
        bad = grad_mismatch(got, want)
        idx = np.argwhere(bad)[:5]
        detail = "; ".join("%s got %.9g ref %.9g" % (tuple(i), got[tuple(i)], want[tuple(i)]) for i in idx)
        assert not bad.any(), "%s %s: %d of %d entries off (max|ref| %.4g): %s" % (
            what, name, bad.sum(), bad.size, np.abs(want).max(), detail)


@pytest.mark.parametrize("flags", [O.G_TEX, O.G_SCORE, O.G_INTERIOR, O.G_EDGE, O.G_ALL])
def test_backward_plain_small(ctx, flags):
    sc = I.plain_small()
    sid, got, (g, col, verts, tex) = gpu_forward(ctx, sc)
    ref = _oracle_fwd(sc)
    gc, sw = upstream(ref, 1)
    rt, rv = O.backward(sc.verts, sc.tex, sc.grid_n, sc.cams, 1, ref, gc, sw, flags=flags)
    gt, gv = gpu_backward(ctx, sid, sc, 1, g, col, gc, sw, flags | 0x100, verts, tex)
    _check_grads(gt, gv, rt, rv, "flags=%d" % flags)


def test_backward_samples_and_reuse(ctx):
    """S = 5 (a full and a ragged group); with and without plan reuse."""
    sc = I.plain_small(soup_seed=8, mask_seed=9)
    S = 5
    sid, got, (g, col, verts, tex) = gpu_forward(ctx, sc, S=S)
    ref = _oracle_fwd(sc, S=S)
    gc, sw = upstream(ref, S, seed=3)
    rt, rv = O.backward(sc.verts, sc.tex, sc.grid_n, sc.cams, S, ref, gc, sw)
    for flags in (O.G_ALL | 0x100, O.G_ALL):
        gt, gv = gpu_backward(ctx, sid, sc, S, g, col, gc, sw, flags, verts, tex)
        _check_grads(gt, gv, rt, rv, "S=5 flags=%x" % flags)


def test_backward_batched_views(ctx):
    sc = I.batched_views()
    sid, got, (g, col, verts, tex) = gpu_forward(ctx, sc)
    ref = _oracle_fwd(sc)
    gc, sw = upstream(ref, 1, seed=5)
    rt, rv = O.backward(sc.verts, sc.tex, sc.grid_n, sc.cams, 1, ref, gc, sw)
    gt, gv = gpu_backward(ctx, sid, sc, 1, g, col, gc, sw, O.G_ALL | 0x100, verts, tex)
    _check_grads(gt, gv, rt, rv, "batched")


def test_backward_edge_cases(ctx):
    sc = _edge_scene()
    sid, got, (g, col, verts, tex) = gpu_forward(ctx, sc, S=3)
    ref = _oracle_fwd(sc, S=3)
    gc, sw = upstream(ref, 3, seed=6)
    rt, rv = O.backward(sc.verts, sc.tex, sc.grid_n, sc.cams, 3, ref, gc, sw)
    gt, gv = gpu_backward(ctx, sid, sc, 3, g, col, gc, sw, O.G_ALL | 0x100, verts, tex)
    _check_grads(gt, gv, rt, rv, "edge cases")


# ------------------------------------------------------------------ full size
def test_large_batch_full_size_sampled_rows(ctx):
    """The 1080p workload at full size (100k triangles, 4x1920x1080 +
    4x960x540, 4 samples) in the bench's launch configuration; the oracle
    recomputes sampled rows of every view, and the backward is checked with
    upstream gradients confined to one row per view."""
    import torch
    sc = I.large_batch()
    S = sc.samples
    sid, got, (g, col, verts, tex) = gpu_forward(ctx, sc, n_front=True)
    rng = np.random.default_rng(99)
    rows = [int(rng.integers(1, c.height - 2)) for c in sc.cams]
    for v, (cam, r) in enumerate(zip(sc.cams, rows)):
        ref = O.forward(sc.verts, sc.tex, sc.grid_n, [cam], sc.seeds[v:v + 1], S=S, bg=sc.bg, rows=(r, r + 1))[0]
        for k in ("tri_id", "n_front", "bary", "depth"):
            assert np.array_equal(got[v][k][:, r], ref[k][:, r]), (v, k)
        assert np.allclose(got[v]["color"][:, :, r], ref["color"][:, :, r], rtol=1e-5, atol=1e-7)
    # backward: upstream non-zero on one row per view only
    gcs, sws, refs = [], [], []
    for v, (cam, r) in enumerate(zip(sc.cams, rows)):
        shape_c, shape_s = got[v]["color"].shape, got[v]["tri_id"].shape
        gc = np.zeros(shape_c, np.float32)
        sw = np.zeros(shape_s, np.float32)
        gc[:, :, r] = rng.standard_normal((S, shape_c[1], shape_c[3]))
        sw[:, r] = rng.uniform(0.1, 1.0, (S, shape_s[2]))
        gcs.append(gc)
        sws.append(sw)
    gt, gv = gpu_backward(ctx, sid, sc, S, g, col, gcs, sws, O.G_ALL | 0x100, verts, tex)
    rt = np.zeros(sc.tex.shape)
    rv = np.zeros(sc.verts.shape)
    for v, (cam, r) in enumerate(zip(sc.cams, rows)):
        # rows r-1 .. r+1: the pairs that touch row r start on row r-1 or r
        f = O.forward(sc.verts, sc.tex, sc.grid_n, [cam], sc.seeds[v:v + 1], S=S, bg=sc.bg, rows=(r - 1, r + 2))[0]
        a, b = O.backward(sc.verts, sc.tex, sc.grid_n, [cam], S, [f], [gcs[v]], [sws[v]], rows=(r - 1, r + 2))
        rt += a
        rv += b
    _check_grads(gt, gv, rt, rv, "full size")


# ------------------------------------------------------------------ API behaviour
def test_invalid_arguments_launch_nothing(ctx):
    import torch
    from paper_2603_27151_gb300 import native as N
    sc = I.plain_small()
    sid = ctx.soup_upload(torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.tex).cuda(), sc.grid_n)
    g, col, _ = N.alloc_outputs(sc.cams, 1, sc.C)
    bad = I.look_at([0, 0, 3.0], 64, 64)
    bad.fx = float("nan")
    with pytest.raises(N.DsError) as e:
        ctx.raster_forward(sid, [bad], sc.seeds, 1, 0, sc.bg, g, col)
    assert e.value.code == -1
    with pytest.raises(N.DsError) as e:
        ctx.raster_forward(sid, sc.cams, sc.seeds, 0, 0, sc.bg, g, col)
    assert e.value.code == -1
    with pytest.raises(N.DsError) as e:
        ctx.raster_forward(12345, sc.cams, sc.seeds, 1, 0, sc.bg, g, col)
    assert e.value.code == -6
    # buffers of the wrong shape are refused before any pointer reaches the library
    with pytest.raises(ValueError):
        ctx.raster_forward(sid, sc.cams, sc.seeds, 2, 0, sc.bg, g, col)          # allocated for S = 1
    with pytest.raises(ValueError):
        ctx.raster_forward(sid, sc.cams, sc.seeds, 1, 0, sc.bg, g, [c[:, :-1].contiguous() for c in col])
    ctx.raster_forward(sid, sc.cams, sc.seeds, 1, 0, sc.bg, g, col)
    with pytest.raises(ValueError):
        ctx.raster_backward(sid, sc.cams, 1, g, col, [torch.zeros_like(c) for c in col], None, N.DS_G_TEX,
                            None, torch.zeros(10, device="cuda"))                  # not the texture's size
    with pytest.raises(ValueError):
        ctx.raster_backward(sid, sc.cams, 1, g, col, [torch.zeros_like(c) for c in col], None, N.DS_G_INTERIOR,
                            torch.zeros(9 * sc.T - 1, device="cuda"), None)        # not 9 T


def test_no_sync_forward_matches_and_reports_capacity(ctx):
    """DS_NO_SYNC reuses the bin capacity of the previous call; overflow is
    reported by ds_ctx_status, never by a fault."""
    import torch
    from paper_2603_27151_gb300 import native as N
    ctx = N.Context(0)          # fresh context: capacity sized by this test only
    sc = I.plain_small()
    sid, ref, _ = gpu_forward(ctx, sc)
    g, col, _ = N.alloc_outputs(sc.cams, 1, sc.C)
    ctx.raster_forward(sid, sc.cams, sc.seeds, 1, N.DS_NO_SYNC, sc.bg, g, col)
    ctx.status()
    tri, _, _ = N.split_gbuf(g[0])
    assert np.array_equal(tri.cpu().numpy(), ref[0]["tri_id"])
    # a much larger soup in no-sync mode overflows the small capacity
    big = I.batched_views()
    sid2 = ctx.soup_upload(torch.from_numpy(big.verts).cuda(), torch.from_numpy(big.tex).cuda(), big.grid_n)
    g2, col2, _ = N.alloc_outputs(big.cams, 1, big.C)
    ctx.raster_forward(sid2, big.cams, big.seeds, 1, N.DS_NO_SYNC, big.bg, g2, col2)
    with pytest.raises(N.DsError) as e:
        ctx.status()
    assert e.value.code == -4
    ctx.status()   # cleared
    ctx.close()


def test_fused_l2_loss_matches_numpy(ctx):
    """ds_loss_l2: per-sample l, dL/dC and score weights against FP64 numpy."""
    import torch
    from paper_2603_27151_gb300 import native as N
    rng = np.random.default_rng(4)
    S, Co = 3, 5
    shapes = [(37, 23), (64, 48)]
    cols = [rng.uniform(0, 1, (S, Co, h, w)).astype(np.float32) for (w, h) in shapes]
    tgts = [rng.uniform(0, 1, (Co, h, w)).astype(np.float32) for (w, h) in shapes]
    dc = [torch.from_numpy(c).cuda() for c in cols]
    dt = [torch.from_numpy(t).cuda() for t in tgts]
    gc = [torch.empty_like(c) for c in dc]
    sw = [torch.empty((S, c.shape[2], c.shape[3]), dtype=torch.float32, device="cuda") for c in dc]
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    N.loss_l2(dc, dt, gc, sw, loss, scale=1.0 / S)
    torch.cuda.synchronize()
    total = 0.0
    for c, t, g, w in zip(cols, tgts, gc, sw):
        d = c.astype(np.float64) - t[None]
        ell = (d ** 2).sum(1)
        total += ell.sum() / S
        assert np.allclose(g.cpu().numpy(), 2 * d / S, rtol=1e-6, atol=1e-7)
        assert np.allclose(w.cpu().numpy(), ell / S, rtol=1e-5, atol=1e-7)
    assert abs(float(loss.item()) - total) <= 1e-5 * total


def test_backward_is_within_tolerance_on_every_run(ctx):
    """The atomics' summation order changes between runs; every run must
    stay within the tolerance (FP64 accumulation)."""
    sc = I.batched_views()
    sid, got, (g, col, verts, tex) = gpu_forward(ctx, sc)
    ref = _oracle_fwd(sc)
    gc, sw = upstream(ref, 1, seed=5)
    rt, rv = O.backward(sc.verts, sc.tex, sc.grid_n, sc.cams, 1, ref, gc, sw)
    for rep in range(5):
        gt, gv = gpu_backward(ctx, sid, sc, 1, g, col, gc, sw, O.G_ALL | 0x100, verts, tex)
        _check_grads(gt, gv, rt, rv, "run %d" % rep)
