"""The autograd.Function and the CUDA-graph-captured training step."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2603_27151_gb300 import inputs as I
from tests.gpu_helpers import grad_mismatch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return t


def _subset_scene(T=256, W=128, H=96, n_views=2):
    """The first T triangles of the 20k-triangle training soup, seen by the
    first n_views of its cameras at a reduced resolution."""
    sc, _ = I.training_setup(T=20_000, T_ref=1000, n_cams=n_views, width=W, height=H)
    rng = np.random.default_rng(17)
    targets = [rng.uniform(0, 1, (sc.C - 1, H, W)).astype(np.float32) for _ in sc.cams]
    return sc.verts[:T].copy(), sc.tex[:T].copy(), sc, targets


def test_autograd_function_equals_the_oracle_backward(torch):
    """loss.backward() through DiffSoupRaster (colour + logp surrogate) gives
    the oracle's Algorithm-A1 gradient for the same masks."""
    from paper_2603_27151_gb300.raster import Rasterizer, render, l2_stochastic_loss
    verts, tex, sc, targets = _subset_scene()
    S = 2
    seeds = I.mask_seeds(31, len(sc.cams))
    v = torch.from_numpy(verts).cuda()
    t = torch.from_numpy(tex).cuda()
    rast = Rasterizer(v, t, sc.grid_n)
    v.requires_grad_(True)
    t.requires_grad_(True)
    colors, logps, _ = render(rast, sc.cams, seeds, S)
    loss = l2_stochastic_loss(colors, logps, [torch.from_numpy(x).cuda() for x in targets], S)
    loss.backward()
    ref = O.forward(verts, tex, sc.grid_n, sc.cams, seeds, S=S, bg=sc.bg)
    gc, sw = [], []
    for f, tg in zip(ref, targets):
        d = f["color"] - tg[None]
        gc.append((2.0 * d / S).astype(np.float32))
        sw.append(((d.astype(np.float64) ** 2).sum(1) / S).astype(np.float32))
    rt, rv = O.backward(verts, tex, sc.grid_n, sc.cams, S, ref, gc, sw)
    for got, want in ((t.grad.cpu().numpy(), rt), (v.grad.cpu().numpy(), rv)):
        assert not grad_mismatch(got, want).any()
    rast.close()


def test_texture_gradient_matches_finite_differences_on_a_256_triangle_subset(torch):
    """Averaged over masks, the autograd gradient of the texture logits equals
    central differences of the closed-form expected loss (Eq. 7)."""
    from paper_2603_27151_gb300.raster import Rasterizer, render, l2_stochastic_loss
    verts, tex, sc, targets = _subset_scene()
    _, eg = O.expected(verts, tex.astype(np.float64), sc.grid_n, sc.cams, targets, bg=sc.bg)
    v = torch.from_numpy(verts).cuda()
    t = torch.from_numpy(tex).cuda()
    rast = Rasterizer(v, t, sc.grid_n)
    t.requires_grad_(True)
    tg = [torch.from_numpy(x).cuda() for x in targets]
    S, reps = 64, 16
    ests = []
    for r in range(reps):
        t.grad = None
        colors, logps, _ = render(rast, sc.cams, I.mask_seeds(100 + r, len(sc.cams)), S)
        l2_stochastic_loss(colors, logps, tg, S).backward()
        ests.append(t.grad.double().cpu().numpy())
    ests = np.array(ests)
    m, se = ests.mean(0), ests.std(0, ddof=1) / math.sqrt(reps)
    # finite differences of E[l] on the logits with the largest expected gradient
    t64 = tex.astype(np.float64)
    order = np.argsort(-np.abs(eg).ravel())[:24]
    h = 1e-5
    for flat in order:
        k = np.unravel_index(flat, tex.shape)
        tp, tm = t64.copy(), t64.copy()
        tp[k] += h
        tm[k] -= h
        fd = (O.expected(verts, tp, sc.grid_n, sc.cams, targets, bg=sc.bg, with_grad=False)[0].sum()
              - O.expected(verts, tm, sc.grid_n, sc.cams, targets, bg=sc.bg, with_grad=False)[0].sum()) / (2 * h)
        assert abs(fd - eg[k]) <= 1e-6 * max(1.0, abs(fd))
        assert abs(m[k] - fd) <= 5 * se[k] + 1e-3 * abs(fd), (k, m[k], fd, se[k])
    rast.close()


def test_captured_training_step(torch):
    """A reduced training workload: the graph replay computes the same loss as
    the eager step for the same views, and training lowers the loss on a
    fixed set of views."""
    from paper_2603_27151_gb300 import native as N
    from paper_2603_27151_gb300.train import TrainStep
    ts = TrainStep(T=2000, T_ref=20_000, n_cams=8, width=256, height=192)

    def eval_loss():
        g, col, _ = N.alloc_outputs(ts.sc.cams, 1, ts.sc.C)
        ts.ctx.raster_forward(ts.sid, ts.sc.cams, I.mask_seeds(5, 8), 1, N.DS_MODE_THRESHOLD_HALF, ts.sc.bg, g, col)
        loss = torch.zeros(1, device="cuda")
        N.loss_l2(col, [ts.targets_all[i] for i in range(8)], None, None, loss)
        torch.cuda.synchronize()
        return float(loss.item())

    before = eval_loss()
    ts.capture()
    # replay vs eager on identical state and views
    state = (ts.verts.clone(), ts.tex.clone())
    ts._load_views(1000)
    ts.graph.replay()
    torch.cuda.synchronize()
    replay_loss = float(ts.loss.item())
    ts.verts.copy_(state[0])
    ts.tex.copy_(state[1])
    ts._load_views(1000)
    ts._body(no_sync=False)
    torch.cuda.synchronize()
    assert abs(float(ts.loss.item()) - replay_loss) <= 1e-6 * abs(replay_loss)
    for _ in range(60):
        ts.step()
    assert ts.check()
    after = eval_loss()
    assert after < 0.9 * before, (before, after)
