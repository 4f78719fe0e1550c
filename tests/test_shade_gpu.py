"""GPU parity of the deferred shading pass (ds_shade_forward / _backward)
against the FP64 oracle (oracle/shading.py) on the same seeded inputs.

Tolerances (FP32 on the GPU against FP64):
  - rgb: |d| <= 1e-5 (values in [0, 1]; a 16-term FP32 dot product per
    layer, three layers and a sigmoid carry a few 1e-7 of rounding);
  - feature gradient: |d| <= 1e-5 (1 + |ref|);
  - parameter gradient: |d| <= 1e-4 (|ref| + 1e-2 max|ref|): per-thread FP32
    partial sums over a CTA's pixels, summed across CTAs in FP64.
"""
import numpy as np
import pytest

from oracle import shading as SH
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


def _params(seed=11):
    rng = np.random.default_rng(seed)
    W1, b1, W2, b2, W3, b3 = SH.unpack(SH.xavier_params(seed))
    # non-zero biases so that both sides of every ReLU occur
    return SH.pack(W1, rng.normal(0, 0.3, 16), W2, rng.normal(0, 0.3, 16), W3, rng.normal(0, 0.3, 3))


def _cams():
    eyes = I.sphere_eyes(3, 3.0, np.random.default_rng(4))
    return [I.look_at(eyes[0], 96, 64), I.look_at(eyes[1], 37, 23), I.look_at(eyes[2], 300, 17)]


def _feats(cams, S, seed=2):
    rng = np.random.default_rng(seed)
    return [rng.uniform(0, 1, (S, 7, c.height, c.width)).astype(np.float32) for c in cams]


def _to(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _run(ctx, cams, params, feats, grads=None, overwrite=True, grad_feat_init=None):
    import torch
    p = _to(params.astype(np.float32))
    f = [_to(x) for x in feats]
    rgb = [torch.empty((x.shape[0], 3, x.shape[2], x.shape[3]), device="cuda") for x in feats]
    ctx.shade_forward(cams, p, f, rgb)
    out = dict(rgb=[r.cpu().numpy() for r in rgb])
    if grads is not None:
        g = [_to(x) for x in grads]
        gf = [torch.zeros_like(x) if grad_feat_init is None else _to(grad_feat_init[i]) for i, x in enumerate(f)]
        gp = torch.zeros_like(p)
        ctx.shade_backward(cams, p, f, g, gf, gp, overwrite=overwrite)
        out.update(gf=[x.cpu().numpy() for x in gf], gp=gp.cpu().numpy())
    torch.cuda.synchronize()
    return out


def _check_gp(got, ref):
    tol = 1e-4 * (np.abs(ref) + 1e-2 * np.abs(ref).max())
    bad = np.abs(got - ref) > tol
    assert not bad.any(), "param grads differ at %s: %s vs %s" % (np.nonzero(bad)[0][:8], got[bad][:4], ref[bad][:4])


@pytest.mark.parametrize("S", [1, 3, 4])
def test_shade_forward_and_backward_small(ctx, S):
    """Three views (96x64, 37x23, 300x17: ragged last blocks of 256 pixels)."""
    cams, params = _cams(), _params()
    feats = _feats(cams, S)
    rng = np.random.default_rng(7)
    grads = [rng.normal(size=(S, 3, c.height, c.width)).astype(np.float32) for c in cams]
    got = _run(ctx, cams, params, feats, grads)
    gp_ref = np.zeros(SH.N_PARAMS)
    for v, c in enumerate(cams):
        ref = SH.shade(feats[v], c, params)
        assert np.abs(got["rgb"][v] - ref).max() <= 1e-5, v
        gf, gp = SH.shade_backward(feats[v], c, params, grads[v])
        assert np.all(np.abs(got["gf"][v] - gf) <= 1e-5 * (1 + np.abs(gf))), v
        gp_ref += gp
    _check_gp(got["gp"], gp_ref)


def test_shade_zero_features_and_saturated_alpha(ctx):
    """A = 1 returns the feature colour exactly and stops the MLP gradient;
    all-zero features (background pixels) give the MLP of the SH alone."""
    cams, params = _cams()[:2], _params(5)
    feats = _feats(cams, 2, seed=9)
    feats[0][:, 3] = 1.0
    feats[1][:] = 0.0
    rng = np.random.default_rng(1)
    grads = [rng.normal(size=(2, 3, c.height, c.width)).astype(np.float32) for c in cams]
    got = _run(ctx, cams, params, feats, grads)
    assert np.array_equal(got["rgb"][0], feats[0][:, 0:3])
    gp_ref = np.zeros(SH.N_PARAMS)
    for v, c in enumerate(cams):
        ref = SH.shade(feats[v], c, params)
        assert np.abs(got["rgb"][v] - ref).max() <= 1e-5
        gf, gp = SH.shade_backward(feats[v], c, params, grads[v])
        assert np.all(np.abs(got["gf"][v] - gf) <= 1e-5 * (1 + np.abs(gf)))
        gp_ref += gp
    _check_gp(got["gp"], gp_ref)


def test_shade_backward_accumulates_and_is_deterministic(ctx):
    import torch
    cams, params = _cams(), _params(3)
    feats = _feats(cams, 2, seed=4)
    rng = np.random.default_rng(8)
    grads = [rng.normal(size=(2, 3, c.height, c.width)).astype(np.float32) for c in cams]
    init = [rng.normal(size=f.shape).astype(np.float32) for f in feats]
    a = _run(ctx, cams, params, feats, grads)
    b = _run(ctx, cams, params, feats, grads)
    assert np.array_equal(a["gp"], b["gp"])               # fixed-order reduction
    c = _run(ctx, cams, params, feats, grads, overwrite=False, grad_feat_init=init)
    for v in range(3):
        assert np.allclose(c["gf"][v], init[v] + a["gf"][v], rtol=1e-6, atol=1e-6)
    # grad_params accumulates too
    p = _to(params.astype(np.float32))
    f = [_to(x) for x in feats]
    g = [_to(x) for x in grads]
    gp = torch.full_like(p, 0.5)
    ctx.shade_backward(cams, p, f, g, None, gp, overwrite=False)
    assert np.allclose(gp.cpu().numpy(), 0.5 + a["gp"], rtol=1e-6, atol=1e-6)


def test_shade_invalid_arguments_and_empty_call(ctx):
    import torch
    from paper_2603_27151_gb300 import native as N
    cams, params = _cams()[:1], _params()
    p = _to(params.astype(np.float32))
    f = [_to(_feats(cams, 1)[0])]
    rgb = [torch.empty((1, 3, 64, 96), device="cuda")]
    with pytest.raises(N.DsError):
        ctx.shade_forward(cams, None, f, rgb)
    bad = I.look_at([0.0, 0.0, 3.0], 96, 64)
    bad.fx = 0.0
    with pytest.raises(N.DsError):
        ctx.shade_forward([bad], p, f, rgb)
    # no views: forward is a no-op, an overwriting backward zeroes grad_params
    ctx.shade_forward([], p, [], [])
    gp = torch.full_like(p, 3.0)
    ctx.shade_backward([], p, [], [], None, gp, overwrite=True)
    torch.cuda.synchronize()
    assert float(gp.abs().max()) == 0.0


def test_shade_autograd_chain_into_the_rasteriser(ctx):
    """Gradients flow from an RGB loss through the shading pass into the
    colour features that the rasteriser's backward consumes."""
    import torch
    from paper_2603_27151_gb300.shade import init_params, shade
    cams = _cams()[:2]
    feats = [_to(x).requires_grad_() for x in _feats(cams, 2, seed=6)]
    params = init_params(3).requires_grad_()
    rgbs = shade(ctx, cams, params, feats)
    loss = sum((r ** 2).sum() for r in rgbs)
    loss.backward()
    for v, c in enumerate(cams):
        gf, gp = SH.shade_backward(feats[v].detach().cpu().numpy(), c, params.detach().cpu().numpy().astype(np.float64),
                                   2.0 * rgbs[v].detach().cpu().numpy())
        assert np.all(np.abs(feats[v].grad.cpu().numpy() - gf) <= 1e-5 * (1 + np.abs(gf)))
    assert params.grad is not None and torch.isfinite(params.grad).all()


# ----------------------------------------------------------- full size
def _crop(cam, x0, y0, w, h):
    """The camera of the window [x0, x0+w) x [y0, y0+h) of ``cam``'s image."""
    return I.Camera(w, h, cam.fx, cam.fy, cam.cx - x0, cam.cy - y0, cam.R, cam.t, cam.near)


def test_shade_full_size_batch(ctx):
    """The 1080p batch (4 x 1920x1080 + 4 x 960x540, S = 4) with the
    rasteriser's own colour features, in one launch.  rgb is checked on
    windows against the oracle; the upstream gradient is zero outside the
    windows, so the exact parameter gradient is the oracle's over the windows
    and the feature gradient is zero elsewhere."""
    import torch
    from paper_2603_27151_gb300 import native as N
    sc = I.large_batch()
    S = sc.samples
    verts, tex = _to(sc.verts), _to(sc.tex)
    sid = ctx.soup_upload(verts, tex, sc.grid_n)
    g, col, _ = N.alloc_outputs(sc.cams, S, sc.C, "cuda", n_front=False)
    ctx.raster_forward(sid, sc.cams, sc.seeds, S, 0, sc.bg, g, col)
    params = _params(21)
    p = _to(params.astype(np.float32))
    rgb = [torch.empty((S, 3, c.height, c.width), device="cuda") for c in sc.cams]
    ctx.shade_forward(sc.cams, p, col, rgb)
    rng = np.random.default_rng(3)
    wins = []
    grads = [torch.zeros_like(r) for r in rgb]
    for v, c in enumerate(sc.cams):
        for (x0, y0) in [(0, 0), (c.width - 40, c.height - 24), (c.width // 2 - 13, c.height // 3)]:
            w, h = 40, 24
            gwin = rng.normal(size=(S, 3, h, w)).astype(np.float32)
            grads[v][:, :, y0:y0 + h, x0:x0 + w] = _to(gwin)
            wins.append((v, x0, y0, w, h, gwin))
    gf = [torch.zeros_like(x) for x in col]
    gp = torch.zeros_like(p)
    ctx.shade_backward(sc.cams, p, col, grads, gf, gp, overwrite=True)
    torch.cuda.synchronize()
    gp_ref = np.zeros(SH.N_PARAMS)
    mask = [np.zeros((c.height, c.width), bool) for c in sc.cams]
    for (v, x0, y0, w, h, gwin) in wins:
        cam = _crop(sc.cams[v], x0, y0, w, h)
        fwin = col[v][:, :, y0:y0 + h, x0:x0 + w].cpu().numpy()
        ref = SH.shade(fwin, cam, params)
        assert np.abs(rgb[v][:, :, y0:y0 + h, x0:x0 + w].cpu().numpy() - ref).max() <= 1e-5, (v, x0, y0)
        gfr, gpr = SH.shade_backward(fwin, cam, params, gwin)
        got = gf[v][:, :, y0:y0 + h, x0:x0 + w].cpu().numpy()
        assert np.all(np.abs(got - gfr) <= 1e-5 * (1 + np.abs(gfr))), (v, x0, y0)
        gp_ref += gpr
        mask[v][y0:y0 + h, x0:x0 + w] = True
    _check_gp(gp.cpu().numpy(), gp_ref)
    for v in range(len(sc.cams)):
        rest = gf[v].cpu().numpy()[:, :, ~mask[v]]
        assert not rest.any(), v
        r = rgb[v].cpu().numpy()
        assert np.isfinite(r).all() and r.min() >= 0.0 and r.max() <= 1.0
    ctx.soup_free(sid)
