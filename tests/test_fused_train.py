"""The fused training pass (ds_raster_train_l2): forward, per-pixel L2 loss
and backward in one call.  It must give the separate calls' results --
G-buffers, colours, upstream gradients and score weights bit for bit (same
arithmetic), gradients up to the order of FP64 summation -- and the
oracle's gradients within the parity tolerance."""
import numpy as np
import pytest

import oracle as O
from paper_2603_27151_gb300 import inputs as I
from tests.gpu_helpers import grad_mismatch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_27151_gb300 import native as N
    return N


def _targets(sc, seed=23):
    rng = np.random.default_rng(seed)
    return [rng.uniform(0, 1, (sc.C - 1, c.height, c.width)).astype(np.float32) for c in sc.cams]


def _buffers(N, sc, S):
    import torch
    g, col, _ = N.alloc_outputs(sc.cams, S, sc.C)
    gc = [torch.empty_like(c) for c in col]
    sw = [torch.empty((S, c.height, c.width), dtype=torch.float32, device="cuda") for c in sc.cams]
    return g, col, gc, sw


def _separate(N, ctx, sid, sc, S, mode, tg, flags, verts, tex):
    import torch
    g, col, gc, sw = _buffers(N, sc, S)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gv, gt = torch.zeros_like(verts), torch.zeros_like(tex)
    ctx.raster_forward(sid, sc.cams, sc.seeds, S, mode, sc.bg, g, col)
    N.loss_l2(col, tg, gc, sw, loss, scale=1.0 / S)
    ctx.raster_backward(sid, sc.cams, S, g, col, gc, sw, flags | N.DS_REUSE_FORWARD | N.DS_OVERWRITE, gv, gt)
    torch.cuda.synchronize()
    return g, col, gc, sw, loss, gv, gt


def _fused(N, ctx, sid, sc, S, mode, tg, flags, verts, tex):
    import torch
    g, col, gc, sw = _buffers(N, sc, S)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gv, gt = torch.full_like(verts, 7.0), torch.full_like(tex, 7.0)   # overwritten
    ctx.train_l2(sid, sc.cams, sc.seeds, S, mode, sc.bg, g, col, tg, gc, sw, 1.0 / S, loss,
                 flags | N.DS_OVERWRITE, gv, gt)
    torch.cuda.synchronize()
    return g, col, gc, sw, loss, gv, gt


def _close(a, b, rtol=1e-6):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    tol = rtol * np.maximum(np.abs(b), 1e-6 * np.abs(b).max())
    return not (np.abs(a - b) > tol).any()


@pytest.mark.parametrize("case", ["batched", "batched_s1", "batched_s5", "threshold", "plain_tile32"])
def test_fused_pass_equals_the_separate_calls(lib, case):
    """S = 1 runs the fully fused kernel, S > 1 the forward-with-loss kernel
    followed by the backward kernel."""
    import torch
    N = lib
    sc = I.plain_small() if case == "plain_tile32" else I.batched_views()
    S = {"batched_s5": 5, "batched_s1": 1}.get(case, 2)
    mode = N.DS_MODE_THRESHOLD_HALF if case == "threshold" else N.DS_MODE_STOCHASTIC
    ctx = N.Context(0)
    if case == "plain_tile32":
        ctx.set_tuning(32, 8, 0, 64)
    verts, tex = torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.tex).cuda()
    sid = ctx.soup_upload(verts, tex, sc.grid_n, borrow=True)
    tg = [torch.from_numpy(x).cuda() for x in _targets(sc)]
    a = _separate(N, ctx, sid, sc, S, mode, tg, N.DS_G_ALL, verts, tex)
    b = _fused(N, ctx, sid, sc, S, mode, tg, N.DS_G_ALL, verts, tex)
    for v in range(len(sc.cams)):
        assert torch.equal(a[0][v], b[0][v]), "G-buffer differs in view %d" % v
        for k, name in ((1, "colour"), (2, "grad_color"), (3, "score_w")):
            assert torch.equal(a[k][v].view(torch.int32), b[k][v].view(torch.int32)), "%s differs in view %d" % (name, v)
    assert abs(float(a[4]) - float(b[4])) <= 1e-5 * abs(float(a[4]))
    assert _close(b[5], a[5]), "vertex gradient differs"
    assert _close(b[6], a[6]), "texture gradient differs"
    ctx.close()


def test_fused_pass_matches_the_oracle(lib):
    import torch
    N = lib
    sc = I.batched_views()
    S = 2
    ctx = N.Context(0)
    verts, tex = torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.tex).cuda()
    sid = ctx.soup_upload(verts, tex, sc.grid_n, borrow=True)
    targets = _targets(sc)
    tg = [torch.from_numpy(x).cuda() for x in targets]
    g, col, gc, sw, loss, gv, gt = _fused(N, ctx, sid, sc, S, N.DS_MODE_STOCHASTIC, tg, N.DS_G_ALL, verts, tex)
    ref = O.forward(sc.verts, sc.tex, sc.grid_n, sc.cams, sc.seeds, S=S, bg=sc.bg)
    rgc, rsw, total = [], [], 0.0
    for f, t in zip(ref, targets):
        d = f["color"].astype(np.float64) - t[None].astype(np.float64)
        ell = (d ** 2).sum(1)
        rgc.append((2.0 * d / S).astype(np.float32))
        rsw.append((ell / S).astype(np.float32))
        total += ell.sum() / S
    for v, f in enumerate(ref):
        tri, _, _ = N.split_gbuf(g[v])
        assert np.array_equal(tri.cpu().numpy(), f["tri_id"])
        assert np.allclose(gc[v].cpu().numpy(), rgc[v], rtol=1e-5, atol=1e-6)
        assert np.allclose(sw[v].cpu().numpy(), rsw[v], rtol=1e-5, atol=1e-6)
    assert abs(float(loss) - total) <= 1e-4 * total
    rt, rv = O.backward(sc.verts, sc.tex, sc.grid_n, sc.cams, S, ref, rgc, rsw)
    assert not grad_mismatch(gt.cpu().numpy(), rt).any()
    assert not grad_mismatch(gv.cpu().numpy(), rv).any()
    ctx.close()


def test_fused_pass_rejects_bad_arguments(lib):
    import torch
    N = lib
    sc = I.plain_small()
    ctx = N.Context(0)
    verts, tex = torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.tex).cuda()
    sid = ctx.soup_upload(verts, tex, sc.grid_n, borrow=True)
    g, col, gc, sw = _buffers(N, sc, 1)
    tg = [torch.zeros((sc.C - 1, 64, 64), device="cuda")]
    loss = torch.zeros(1, device="cuda")
    with pytest.raises(N.DsError) as e:
        ctx.train_l2(sid, sc.cams, sc.seeds, 1, 0, sc.bg, g, col, tg, gc, sw, float("nan"), loss, N.DS_G_ALL)
    assert e.value.code == -1
    with pytest.raises(N.DsError) as e:
        ctx.train_l2(sid, sc.cams, sc.seeds, 1, 0, sc.bg, g, col, tg, gc, sw, 1.0, loss, N.DS_G_ALL | 0x100)
    assert e.value.code == -1
    ctx.close()
