"""GPU parity of the multi-resolution feature grids against the oracle
(or_compose / or_restrict / or_resample) on the same seeded inputs.

The composition decides visibility (through the opacity), so it runs in FP32
in the same order on both sides and must match bit for bit, like the
activation and the rasteriser's visibility.  The level gradients are the
adjoint of the composition applied to the FP64 texture gradient: within
1e-4 of the oracle (the GPU restricts in FP32, the oracle in FP64)."""
import numpy as np
import pytest

import oracle as O
from paper_2603_27151_gb300 import inputs as I
from tests.gpu_helpers import assert_forward_equal, grad_mismatch, upstream

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


def _flat(levels):
    import torch
    return torch.from_numpy(np.concatenate([l.reshape(-1) for l in levels])).cuda()


@pytest.mark.parametrize("r_min,r_max,C", [(2, 5, 8), (0, 3, 4), (1, 2, 3), (3, 3, 8), (0, 5, 16)])
def test_compose_bit_exact(ctx, r_min, r_max, C):
    import torch
    from paper_2603_27151_gb300 import native as N
    T = 37
    lv = I.level_logits(T, r_min, r_max, C, np.random.default_rng(r_min * 10 + r_max))
    ref = O.compose(lv, r_min, r_max)
    out = torch.empty((T, N.level_V(r_max), C), device="cuda")
    N.levels_compose(_flat(lv), T, r_min, r_max, C, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)
    N.levels_compose(_flat(lv), T, r_min, r_max, C, out, activate=True)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), O.activate(ref))


@pytest.mark.parametrize("r_src,r_dst", [(2, 5), (5, 2), (3, 3), (0, 4), (4, 1)])
def test_resample_bit_exact(ctx, r_src, r_dst):
    import torch
    from paper_2603_27151_gb300 import native as N
    T, C = 23, 5
    src = np.random.default_rng(r_src + 7 * r_dst).standard_normal((T, N.level_V(r_src), C)).astype(np.float32)
    dst = torch.empty((T, N.level_V(r_dst), C), device="cuda")
    N.levels_resample(torch.from_numpy(src).cuda(), T, r_src, C, dst, r_dst)
    torch.cuda.synchronize()
    assert np.array_equal(dst.cpu().numpy(), O.resample(src, r_src, r_dst))


def _render_levels(ctx, sc, lv, r_min, r_max, S):
    import torch
    from paper_2603_27151_gb300 import native as N
    verts = torch.from_numpy(sc.verts).cuda()
    tex = _flat(lv)
    sid = ctx.soup_upload_levels(verts, tex, sc.T, r_min, r_max, sc.C)
    g, col, nf = N.alloc_outputs(sc.cams, S, sc.C, "cuda", n_front=True)
    ctx.raster_forward(sid, sc.cams, sc.seeds, S, 0, sc.bg, g, col, nf)
    torch.cuda.synchronize()
    got = []
    for v in range(len(sc.cams)):
        tri, bary, depth = N.split_gbuf(g[v])
        got.append(dict(tri_id=tri.cpu().numpy(), bary=bary.cpu().numpy(), depth=depth.cpu().numpy(),
                        color=col[v].cpu().numpy(), n_front=nf[v].cpu().numpy()))
    return sid, got, (g, col, verts, tex)


@pytest.mark.parametrize("r_min,r_max,S", [(2, 5, 1), (0, 3, 3)])
def test_level_soup_forward_and_backward(ctx, r_min, r_max, S):
    import torch
    from paper_2603_27151_gb300 import native as N
    sc, lv = I.levels_scene(r_min=r_min, r_max=r_max)
    sid, got, (g, col, verts, tex) = _render_levels(ctx, sc, lv, r_min, r_max, S)
    ref = O.forward_levels(sc.verts, lv, r_min, r_max, sc.cams, sc.seeds, S=S, bg=sc.bg)
    assert_forward_equal(got, ref)
    gc, sw = upstream(ref, S, seed=4)
    gt = torch.zeros_like(tex)
    gv = torch.zeros_like(verts)
    ctx.raster_backward(sid, sc.cams, S, g, col, [torch.from_numpy(x).cuda() for x in gc],
                        [torch.from_numpy(x).cuda() for x in sw], N.DS_G_ALL | N.DS_REUSE_FORWARD, gv, gt)
    torch.cuda.synchronize()
    gl_ref, gv_ref = O.backward_levels(sc.verts, lv, r_min, r_max, sc.cams, S, ref, gc, sw)
    got_levels = N.split_levels(gt, sc.T, r_min, r_max, sc.C)
    for R, a, b in zip(range(r_min, r_max + 1), got_levels, gl_ref):
        bad = grad_mismatch(a.cpu().numpy(), b)
        assert not bad.any(), "level %d: %d of %d entries differ" % (R, bad.sum(), bad.size)
    bad = grad_mismatch(gv.cpu().numpy(), gv_ref)
    assert bad.mean() < 1e-3
    # accumulate mode adds to what is there
    gt2 = gt.clone()
    ctx.raster_backward(sid, sc.cams, S, g, col, [torch.from_numpy(x).cuda() for x in gc],
                        [torch.from_numpy(x).cuda() for x in sw], N.DS_G_TEX | N.DS_G_SCORE | N.DS_REUSE_FORWARD,
                        None, gt2)
    torch.cuda.synchronize()
    assert torch.allclose(gt2, 2 * gt, rtol=1e-5, atol=1e-7)
    ctx.soup_free(sid)


def test_single_level_soup_equals_plain_soup(ctx):
    """r_min = r_max: the level soup is the plain soup of that grid."""
    import torch
    from paper_2603_27151_gb300 import native as N
    sc, lv = I.levels_scene(r_min=3, r_max=3, T=500, res=((96, 80),))
    sid_l, got_l, (g_l, col_l, verts, tex) = _render_levels(ctx, sc, lv, 3, 3, 2)
    sid_p = ctx.soup_upload(verts, tex.view(sc.T, -1, sc.C).contiguous(), 8)
    g, col, nf = N.alloc_outputs(sc.cams, 2, sc.C, "cuda", n_front=True)
    ctx.raster_forward(sid_p, sc.cams, sc.seeds, 2, 0, sc.bg, g, col, nf)
    torch.cuda.synchronize()
    assert torch.equal(g[0], g_l[0]) and torch.equal(col[0], col_l[0])


def test_fused_training_pass_on_a_level_soup(ctx):
    """The fused forward + L2 + backward pass returns the same level
    gradients as the separate calls."""
    import torch
    from paper_2603_27151_gb300 import native as N
    sc, lv = I.levels_scene(r_min=2, r_max=4, T=800, res=((128, 96), (64, 64)))
    S = 2
    sid, got, (g, col, verts, tex) = _render_levels(ctx, sc, lv, 2, 4, S)
    rng = np.random.default_rng(5)
    targets = [torch.from_numpy(rng.uniform(0, 1, (sc.C - 1, c.height, c.width)).astype(np.float32)).cuda()
               for c in sc.cams]
    gcol = [torch.empty_like(c) for c in col]
    sw = [torch.empty((S, c.height, c.width), device="cuda") for c in sc.cams]
    loss = torch.zeros(1, device="cuda")
    N.loss_l2(col, targets, gcol, sw, loss, scale=1.0 / S)
    gt_a, gv_a = torch.zeros_like(tex), torch.zeros_like(verts)
    ctx.raster_backward(sid, sc.cams, S, g, col, gcol, sw, N.DS_G_ALL | N.DS_REUSE_FORWARD, gv_a, gt_a)
    gt_b, gv_b = torch.zeros_like(tex), torch.zeros_like(verts)
    loss_b = torch.zeros(1, device="cuda")
    ctx.train_l2(sid, sc.cams, sc.seeds, S, N.DS_MODE_STOCHASTIC, sc.bg, g, col, targets, gcol, sw, 1.0 / S, loss_b,
                 N.DS_G_ALL | N.DS_OVERWRITE, gv_b, gt_b)
    torch.cuda.synchronize()
    assert torch.allclose(loss, loss_b, rtol=1e-5)
    a, b = gt_a.cpu().numpy(), gt_b.cpu().numpy()
    assert not grad_mismatch(b, a, rtol=1e-4).any()
    ctx.soup_free(sid)


def test_coarse_to_fine_switch(ctx):
    """The coarse grid's colour features land on the new r_min level (sampled
    at its vertices), the other levels are zero, opacity logits are reset."""
    import torch
    from paper_2603_27151_gb300 import levels as L
    from paper_2603_27151_gb300 import native as N
    T, C = 19, 8
    coarse = np.random.default_rng(2).standard_normal((T, N.level_V(3), C)).astype(np.float32)
    out = L.coarse_to_fine(torch.from_numpy(coarse).cuda(), 3, 2, 5)
    torch.cuda.synchronize()
    parts = [p.cpu().numpy() for p in N.split_levels(out, T, 2, 5, C)]
    ref = O.resample(coarse, 3, 2)
    ref[:, :, C - 1] = 0.0
    assert np.array_equal(parts[0], ref)
    assert all(not p.any() for p in parts[1:])
    fine = L.compose(out, T, 2, 5, C, activate=False)
    assert np.array_equal(fine.cpu().numpy(), O.compose([ref] + [np.zeros_like(p) for p in parts[1:]], 2, 5))
