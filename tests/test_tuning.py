"""Launch-parameter tuning (tile shape, depth bits of the bin key, staging
chunk, CTAs per SM) changes only the work decomposition: for every setting
the forward must equal the oracle bit for bit and the backward must stay
within tolerance of the oracle's estimator; the autotuner must return a
valid setting and leave correct outputs."""
import functools

import numpy as np
import pytest

import oracle as O
from paper_2603_27151_gb300 import inputs as I
from tests.gpu_helpers import assert_forward_equal, gpu_backward, gpu_forward, grad_mismatch, upstream

pytestmark = pytest.mark.gpu

S = 2


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


@functools.lru_cache(maxsize=1)
def _reference():
    sc = I.batched_views()
    ref = O.forward(sc.verts, sc.tex, sc.grid_n, sc.cams, sc.seeds, S=S, bg=sc.bg)
    gc, sw = upstream(ref, S, seed=21)
    rt, rv = O.backward(sc.verts, sc.tex, sc.grid_n, sc.cams, S, ref, gc, sw)
    return sc, ref, gc, sw, rt, rv


@pytest.mark.parametrize("tuning", [(8, -1, 0, 256), (32, -1, 0, 256), (16, 0, 0, 256), (16, 8, 2, 64),
                                    (32, 8, 3, 128), (8, 4, 1, 32)])
def test_every_tuning_gives_the_oracle_result(ctx, tuning):
    sc, ref, gc, sw, rt, rv = _reference()
    ctx.set_tuning(*tuning)
    try:
        assert ctx.get_tuning() == dict(zip(("tile_w", "depth_bits", "blocks_per_sm", "chunk"), tuning))
        sid, got, (g, col, verts, tex) = gpu_forward(ctx, sc, S=S)
        assert_forward_equal(got, ref)
        gt, gv = gpu_backward(ctx, sid, sc, S, g, col, gc, sw, O.G_ALL | 0x100, verts, tex)
        assert not grad_mismatch(gt, rt).any(), "texture gradient off with tuning %s" % (tuning,)
        assert not grad_mismatch(gv, rv).any(), "vertex gradient off with tuning %s" % (tuning,)
        ctx.soup_free(sid)
    finally:
        ctx.set_tuning()


def test_invalid_tunings_are_rejected(ctx):
    from paper_2603_27151_gb300 import native as N
    for bad in [(12, -1, 0, 256), (16, 17, 0, 256), (16, -2, 0, 256), (16, -1, 9, 256), (16, -1, 0, 48),
                (16, -1, 0, 512)]:
        with pytest.raises(N.DsError) as e:
            ctx.set_tuning(*bad)
        assert e.value.code == -1
    assert ctx.get_tuning() == {"tile_w": 16, "depth_bits": -1, "blocks_per_sm": 0, "chunk": 256}


def test_autotune_returns_a_valid_setting_and_correct_outputs(ctx, tmp_path):
    import torch
    from paper_2603_27151_gb300 import autotune, native as N
    sc, ref, gc, sw, rt, rv = _reference()
    verts, tex = torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.tex).cuda()
    sid = ctx.soup_upload(verts, tex, sc.grid_n)
    g, col, _ = N.alloc_outputs(sc.cams, S, sc.C)
    gcd = [torch.from_numpy(x).cuda() for x in gc]
    swd = [torch.from_numpy(x).cuda() for x in sw]
    gv, gt = torch.zeros_like(verts), torch.zeros_like(tex)
    path = str(tmp_path / "tune.json")
    t1 = autotune.tuned(ctx, sid, sc.T, sc.grid_n, sc.C, sc.cams, sc.seeds, S, N.DS_MODE_STOCHASTIC, sc.bg, g, col,
                        gcd, swd, gv, gt, reps=1, path=path)
    assert not t1["cached"] and t1["tile_w"] in (8, 16, 32) and t1["chunk"] in (64, 128, 256)
    torch.cuda.synchronize()
    for v in range(len(sc.cams)):
        tri, bary, depth = N.split_gbuf(g[v])
        assert np.array_equal(tri.cpu().numpy(), ref[v]["tri_id"])
        assert np.array_equal(depth.cpu().numpy(), ref[v]["depth"])
    assert not grad_mismatch(gt.cpu().numpy(), rt).any()
    assert not grad_mismatch(gv.cpu().numpy(), rv).any()
    ctx.set_tuning()
    t2 = autotune.tuned(ctx, sid, sc.T, sc.grid_n, sc.C, sc.cams, sc.seeds, S, N.DS_MODE_STOCHASTIC, sc.bg, g, col,
                        gcd, swd, gv, gt, reps=1, path=path)
    assert t2["cached"] and {k: t2[k] for k in ("tile_w", "depth_bits", "blocks_per_sm", "chunk")} == \
        ctx.get_tuning()
    ctx.soup_free(sid)
    ctx.set_tuning()


def test_autotune_of_the_fused_training_pass(ctx, tmp_path):
    """With targets the autotuner times ds_raster_train_l2; the tuning it
    returns is valid and the outputs of its last run equal the oracle's
    visibility."""
    import torch
    from paper_2603_27151_gb300 import autotune, native as N
    sc, ref, gc, sw, rt, rv = _reference()
    verts, tex = torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.tex).cuda()
    sid = ctx.soup_upload(verts, tex, sc.grid_n)
    g, col, _ = N.alloc_outputs(sc.cams, S, sc.C)
    tg = [torch.rand((sc.C - 1, c.height, c.width), device="cuda") for c in sc.cams]
    gcd = [torch.empty_like(c) for c in col]
    swd = [torch.empty((S, c.height, c.width), device="cuda") for c in sc.cams]
    gv, gt = torch.zeros_like(verts), torch.zeros_like(tex)
    t = autotune.tuned(ctx, sid, sc.T, sc.grid_n, sc.C, sc.cams, sc.seeds, S, N.DS_MODE_STOCHASTIC, sc.bg, g, col,
                       gcd, swd, gv, gt, reps=1, path=str(tmp_path / "tune.json"), targets=tg, scale=1.0 / S)
    assert not t["cached"] and t["tile_w"] in (8, 16, 32)
    torch.cuda.synchronize()
    for v in range(len(sc.cams)):
        tri, _, depth = N.split_gbuf(g[v])
        assert np.array_equal(tri.cpu().numpy(), ref[v]["tri_id"])
        assert np.array_equal(depth.cpu().numpy(), ref[v]["depth"])
    ctx.soup_free(sid)
    ctx.set_tuning()
