"""GPU parity of the fused lambda L1 + (1 - lambda) SSIM loss
(ds_loss_l1_ssim) against the FP64 oracle (oracle/ssim.py).

Tolerances (FP32 moments against FP64): the variance m2 - m1^2 of values in
[0, 1] carries a few 2^-24 of absolute rounding, which SSIM divides by
sigma^2 + C2 >= C2 = 9e-4; the per-pixel loss is therefore checked to
1e-4 absolute and the gradient (derivative maps up to ~1/C2 in flat regions,
blurred) to 1e-3 of its largest magnitude plus 1e-3 relative."""
import numpy as np
import pytest

from oracle import ssim as SS
from paper_2603_27151_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return "cuda"


def _run(colors, targets, scale, lam=0.8):
    import torch
    from paper_2603_27151_gb300 import native as N
    c = [torch.from_numpy(x.astype(np.float32)).cuda() for x in colors]
    t = [torch.from_numpy(x.astype(np.float32)).cuda() for x in targets]
    g = [torch.empty_like(x) for x in c]
    sw = [torch.empty((x.shape[0], x.shape[2], x.shape[3]), device="cuda") for x in c]
    loss = torch.zeros(1, device="cuda")
    N.loss_l1_ssim(c, t, g, sw, loss, lam=lam, scale=scale)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in g], [x.cpu().numpy() for x in sw], float(loss)


def _check(got_g, got_sw, colors, targets, scale, lam=0.8, win=None):
    total = 0.0
    for v, (x, y) in enumerate(zip(colors, targets)):
        ell, g = SS.loss(x.astype(np.float64), y.astype(np.float64), lam=lam)
        a, b = got_sw[v], scale * ell
        ga, gb = got_g[v], scale * g
        if win is not None:
            sl = win[v]
            a, b, ga, gb = a[..., sl[0], sl[1]], b[..., sl[0], sl[1]], ga[..., sl[0], sl[1]], gb[..., sl[0], sl[1]]
        assert np.abs(a - b).max() <= 1e-4 * abs(scale), (v, float(np.abs(a - b).max()))
        tol = 1e-3 * np.abs(gb).max() + 1e-3 * np.abs(gb)
        assert np.all(np.abs(ga - gb) <= tol), (v, float(np.abs(ga - gb).max()), float(np.abs(gb).max()))
        total += float(b.sum())
    return total


@pytest.mark.parametrize("C,S", [(4, 2), (8, 1), (2, 3)])
def test_l1_ssim_small(dev, C, S):
    """Views 70x45, 33x17 (smaller than a tile) and 64x32 (exact tiles)."""
    rng = np.random.default_rng(C * 10 + S)
    sizes = [(70, 45), (33, 17), (64, 32)]
    colors = [rng.uniform(0, 1, (S, C - 1, h, w)) for (w, h) in sizes]
    targets = [rng.uniform(0, 1, (C - 1, h, w)) for (w, h) in sizes]
    g, sw, loss = _run(colors, targets, 0.5)
    total = _check(g, sw, colors, targets, 0.5)
    assert abs(loss - total) <= 1e-4 * abs(total)


def test_l1_ssim_smooth_and_equal_images(dev):
    """Flat and smooth images (the worst case for the variance's rounding)
    and identical images (zero loss and gradient away from ties)."""
    h, w = 40, 50
    yy, xx = np.mgrid[0:h, 0:w]
    smooth = 0.5 + 0.2 * np.sin(xx / 9.0) * np.cos(yy / 7.0)
    colors = [np.stack([smooth, 0.9 * smooth])[:, None].repeat(3, 1), np.full((2, 3, h, w), 0.25)]
    targets = [np.repeat(smooth[None], 3, 0) + 0.01, np.full((3, h, w), 0.3)]
    g, sw, loss = _run(colors, targets, 1.0)
    _check(g, sw, colors, targets, 1.0)
    g, sw, loss = _run([colors[0][:1]], [colors[0][0]], 1.0)
    assert np.abs(sw[0]).max() <= 1e-5 and abs(loss) <= 1e-5 * h * w


def test_l1_ssim_full_size_windows(dev):
    """The 1080p batch (4 x 1920x1080 + 4 x 960x540, S = 4, 7 channels) with
    the rasteriser's colours against synthetic targets, in one launch; the
    oracle checks 48x24 windows (corners and centre) on crops with a 10-pixel
    margin, which hold every pixel the windows depend on."""
    import torch
    from paper_2603_27151_gb300 import native as N
    sc = I.large_batch()
    S = sc.samples
    ctx = N.Context(0)
    sid = ctx.soup_upload(torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.tex).cuda(), sc.grid_n)
    gb, col, _ = N.alloc_outputs(sc.cams, S, sc.C, "cuda")
    ctx.raster_forward(sid, sc.cams, sc.seeds, S, 0, sc.bg, gb, col)
    gen = torch.Generator(device="cuda").manual_seed(3)
    tg = [torch.rand((sc.C - 1, c.height, c.width), generator=gen, device="cuda") for c in sc.cams]
    g = [torch.empty_like(x) for x in col]
    sw = [torch.empty((S, c.height, c.width), device="cuda") for c in sc.cams]
    loss = torch.zeros(1, device="cuda")
    N.loss_l1_ssim(col, tg, g, sw, loss, scale=1.0 / S)
    torch.cuda.synchronize()
    assert abs(float(loss) - sum(float(x.double().sum()) for x in sw)) <= 1e-4 * float(loss)
    for v, c in enumerate(sc.cams):
        for (x0, y0) in [(0, 0), (c.width - 48, c.height - 24), (c.width // 2 - 7, c.height // 2 + 3)]:
            cx0, cy0 = max(0, x0 - 10), max(0, y0 - 10)
            cx1, cy1 = min(c.width, x0 + 58), min(c.height, y0 + 34)
            xc = col[v][:, :, cy0:cy1, cx0:cx1].cpu().numpy()
            yc = tg[v][:, cy0:cy1, cx0:cx1].cpu().numpy()
            ell, gr = SS.loss(xc.astype(np.float64), yc.astype(np.float64))
            sl = (slice(y0 - cy0, y0 - cy0 + 24), slice(x0 - cx0, x0 - cx0 + 48))
            a = sw[v][:, y0:y0 + 24, x0:x0 + 48].cpu().numpy()
            assert np.abs(a - ell[:, sl[0], sl[1]] / S).max() <= 1e-4 / S
            ga = g[v][:, :, y0:y0 + 24, x0:x0 + 48].cpu().numpy()
            gb_ = gr[:, :, sl[0], sl[1]] / S
            assert np.all(np.abs(ga - gb_) <= 1e-3 * np.abs(gb_).max() + 1e-3 * np.abs(gb_))
    ctx.close()
