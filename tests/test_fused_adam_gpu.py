"""ds_raster_backward_adam: the texture's Adam step (Sec. 3.4; supplementary
"Hyperparameters") fused into the backward's gradient finish, against
ds_raster_backward (DS_OVERWRITE) followed by ds_adam_step on the same inputs.

Both apply the same per-value roundings to the same FP32 gradient, so the
texture, m and v agree bit for bit wherever the two backward passes produce
the same FP32 gradient.  The gradients are FP64 atomic sums whose order
varies between runs; a value whose sum rounds to a neighbouring float is
possible but rare, so the test requires all but a few values per million to
be identical and every value to agree to 1e-6 relative.  The vertex
gradients are the same call's."""
import numpy as np
import pytest

from paper_2603_27151_gb300 import inputs as I

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


def _inputs(levels: bool):
    if levels:
        sc, lv = I.levels_scene(r_min=2, r_max=4, T=600)
        tex = np.concatenate([l.reshape(-1) for l in lv]).astype(np.float32)
        return sc, tex, (2, 4)
    sc = I.batched_views()
    return sc, sc.tex.reshape(-1).astype(np.float32), None


def _upload(ctx, sc, verts, tex, lv):
    if lv is None:
        return ctx.soup_upload(verts, tex.view(sc.T, -1, sc.C), sc.grid_n, borrow=True)
    return ctx.soup_upload_levels(verts, tex, sc.T, lv[0], lv[1], sc.C, borrow=True)


def _close(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    same = a == b
    assert (~same).mean() <= 1e-5, (~same).sum()
    assert np.all(np.abs(a - b) <= 1e-6 * np.maximum(np.abs(b), 1e-6)), float(np.abs(a - b).max())


@pytest.mark.parametrize("levels", [False, True])
@pytest.mark.parametrize("step", [1, 7])
def test_fused_adam_equals_backward_then_adam(ctx, levels, step):
    import torch
    from paper_2603_27151_gb300 import native as N
    sc, tex0, lv = _inputs(levels)
    S = 2
    verts = torch.from_numpy(np.ascontiguousarray(sc.verts)).cuda()
    gen = torch.Generator(device="cuda").manual_seed(3)
    m0 = 0.01 * torch.randn(tex0.size, generator=gen, device="cuda")
    v0 = torch.rand(tex0.size, generator=gen, device="cuda") * 1e-3
    flags = N.DS_G_ALL | N.DS_REUSE_FORWARD
    out = {}
    for fused in (False, True):
        tex = torch.from_numpy(tex0).cuda()
        m, v = m0.clone(), v0.clone()
        sid = _upload(ctx, sc, verts, tex, lv)
        g, col, _ = N.alloc_outputs(sc.cams, S, sc.C, "cuda")
        ctx.raster_forward(sid, sc.cams, sc.seeds, S, 0, sc.bg, g, col)
        rng = np.random.default_rng(5)
        gc = [torch.from_numpy(rng.standard_normal(c.shape).astype(np.float32)).cuda() for c in col]
        sw = [torch.from_numpy(rng.uniform(0.1, 1.0, (S, c.height, c.width)).astype(np.float32)).cuda()
              for c in sc.cams]
        gv = torch.zeros_like(verts)
        if fused:
            ctx.raster_backward_adam(sid, sc.cams, S, g, col, gc, sw, flags | N.DS_OVERWRITE, m, v, 0.05, step,
                                     grad_verts=gv)
        else:
            gt = torch.empty_like(tex)
            ctx.raster_backward(sid, sc.cams, S, g, col, gc, sw, flags | N.DS_OVERWRITE, gv, gt)
            N.adam_step(tex, gt, m, v, 0.05, step)
        torch.cuda.synchronize()
        ctx.status()
        ctx.soup_free(sid)
        out[fused] = (tex, m, v, gv)
    assert not torch.equal(out[True][0], torch.from_numpy(tex0).cuda())   # the step moved the texture
    for a, b in zip(out[True], out[False]):
        _close(a, b)


def test_fused_adam_invalid_arguments(ctx):
    import ctypes
    import torch
    from paper_2603_27151_gb300 import native as N
    sc = I.plain_small()
    verts = torch.from_numpy(np.ascontiguousarray(sc.verts)).cuda()
    tex = torch.from_numpy(np.ascontiguousarray(sc.tex)).cuda()
    m, v = torch.zeros_like(tex), torch.zeros_like(tex)
    g, col, _ = N.alloc_outputs(sc.cams, 1, sc.C, "cuda")
    sid = ctx.soup_upload(verts, tex, sc.grid_n, borrow=True)
    ctx.raster_forward(sid, sc.cams, sc.seeds, 1, 0, sc.bg, g, col)
    gc = [torch.ones_like(c) for c in col]
    with pytest.raises(N.DsError):   # step < 1
        ctx.raster_backward_adam(sid, sc.cams, 1, g, col, gc, None, N.DS_G_TEX, m, v, 0.01, 0)
    with pytest.raises(N.DsError):   # no texture term selected
        ctx.raster_backward_adam(sid, sc.cams, 1, g, col, gc, None, N.DS_G_INTERIOR, m, v, 0.01, 1)
    with pytest.raises(N.DsError):   # beta1 out of range
        ctx.raster_backward_adam(sid, sc.cams, 1, g, col, gc, None, N.DS_G_TEX, m, v, 0.01, 1, beta1=1.0)
    L = N.load()
    fwd = (N.ds_view_out * 1)()
    gin = (N.ds_view_gin * 1)()
    fwd[0].gbuf = g[0].data_ptr()
    fwd[0].color = col[0].data_ptr()
    gin[0].grad_color = gc[0].data_ptr()
    with pytest.raises(N.DsError):   # m and v of the wrong size
        ctx.raster_backward_adam(sid, sc.cams, 1, g, col, gc, None, N.DS_G_TEX, m[:-1].contiguous(),
                                 v[:-1].contiguous(), 0.01, 1)
    bad = N.ds_adam_args(None, v.data_ptr(), v.numel(), 0.01, 0.9, 0.999, 1e-8, 1)   # NULL m
    assert L.ds_raster_backward_adam(ctx.h, sid, N.cameras(sc.cams), 1, 1, fwd, gin, N.DS_G_TEX, None,
                                     ctypes.byref(bad), None) == -1
    assert L.ds_raster_backward_adam(ctx.h, sid, N.cameras(sc.cams), 1, 1, fwd, gin, N.DS_G_TEX, None,
                                     None, None) == -1
    ctx.soup_free(sid)
    sid = ctx.soup_upload(verts, tex, sc.grid_n, static=True)
    ctx.raster_forward(sid, sc.cams, sc.seeds, 1, 0, sc.bg, g, col)
    with pytest.raises(N.DsError):   # a static soup cannot be updated
        ctx.raster_backward_adam(sid, sc.cams, 1, g, col, gc, None, N.DS_G_TEX, m, v, 0.01, 1)
    ctx.soup_free(sid)
    torch.cuda.synchronize()
    ctx.status()


def test_fused_adam_level_soup_needs_four_channel_groups(ctx):
    """The level soups' fused update moves four values per access: a level
    soup whose channel count is not a multiple of 4 is refused up front."""
    import torch
    from paper_2603_27151_gb300 import native as N
    rng = np.random.default_rng(8)
    T, C = 50, 3
    verts = torch.from_numpy(I.box_soup(T, 0.3, rng)).cuda()
    tex = torch.from_numpy(np.concatenate([l.reshape(-1) for l in I.level_logits(T, 0, 2, C, rng)])).cuda()
    sid = ctx.soup_upload_levels(verts, tex, T, 0, 2, C, borrow=True)
    cams = [I.look_at([0.0, 0.0, 3.0], 32, 32)]
    g, col, _ = N.alloc_outputs(cams, 1, C, "cuda")
    ctx.raster_forward(sid, cams, [1], 1, 0, np.zeros(C - 1, np.float32), g, col)
    m, v = torch.zeros_like(tex), torch.zeros_like(tex)
    with pytest.raises(N.DsError) as e:
        ctx.raster_backward_adam(sid, cams, 1, g, col, [torch.ones_like(c) for c in col], None, N.DS_G_TEX, m, v,
                                 0.01, 1)
    assert e.value.code == -1
    ctx.soup_free(sid)
    torch.cuda.synchronize()
    ctx.status()
