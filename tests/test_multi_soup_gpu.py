"""Views of different soups in one launch (ds_raster_forward_multi) and the
render server's mixed-soup batches.

A view's pixels depend only on its own soup, camera and seed, so every
output of a multi-soup forward -- triangle ids (indices into the view's own
soup), barycentrics, depths, n_front, colours -- must be bit-identical to the
view rendered alone with ds_raster_forward, and equal the oracle on small
soups; a server batch that mixes soups must give each request the bits it
gets alone."""
import numpy as np
import pytest

import oracle as O
from paper_2603_27151_gb300 import inputs as I
from tests.gpu_helpers import assert_forward_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_27151_gb300 import native as N
    return N


def _soups(n, T0=300, seed=70):
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed + i)
        T = T0 + 137 * i
        out.append((I.box_soup(T, I.edge_length_for(T) * 3.0, rng), I.logits(T, 4, 4, rng)))
    return out


@pytest.mark.parametrize("S,mode", [(1, 0), (3, 0), (2, 1)])
def test_multi_soup_forward_equals_each_view_alone(N, S, mode):
    import torch
    soups = _soups(3)
    ctx = N.Context(0)
    sids = [ctx.soup_upload(torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda(), 4) for v, t in soups]
    eyes = I.sphere_eyes(6, 3.0, np.random.default_rng(5))
    res = [(64, 48), (37, 23), (96, 96), (50, 70), (128, 32), (33, 33)]
    cams = [I.look_at(e, w, h) for e, (w, h) in zip(eyes, res)]
    which = [0, 1, 2, 1, 0, 2]
    seeds = I.mask_seeds(17, len(cams))
    bg = np.array([0.1, 0.2, 0.3], np.float32)
    g, col, nf = N.alloc_outputs(cams, S, 4, "cuda", n_front=True)
    for t in g:
        t.fill_(-7)
    ctx.raster_forward_multi([sids[k] for k in which], cams, seeds, S, mode, bg, g, col, nf)
    torch.cuda.synchronize()
    for v, cam in enumerate(cams):
        ga, ca, fa = N.alloc_outputs([cam], S, 4, "cuda", n_front=True)
        ctx.raster_forward(sids[which[v]], [cam], seeds[v:v + 1], S, mode, bg, ga, ca, fa)
        torch.cuda.synchronize()
        assert torch.equal(g[v], ga[0]), v
        assert torch.equal(nf[v], fa[0]), v
        assert torch.equal(col[v].view(torch.int32), ca[0].view(torch.int32)), v
    # and the oracle, on the first two views
    for v in range(2):
        verts, tex = soups[which[v]]
        ref = O.forward(verts, tex, 4, [cams[v]], seeds[v:v + 1], S=S, mode=mode, bg=bg)
        tri, bary, depth = N.split_gbuf(g[v])
        got = [dict(tri_id=tri.cpu().numpy(), bary=bary.cpu().numpy(), depth=depth.cpu().numpy(),
                    color=col[v].cpu().numpy(), n_front=nf[v].cpu().numpy())]
        assert_forward_equal(got, ref)
    ctx.close()


def test_multi_soup_forward_rejects_mismatched_texture_shapes(N):
    import torch
    (v0, t0), = _soups(1)
    rng = np.random.default_rng(3)
    v1, t1 = I.box_soup(100, 0.3, rng), I.logits(100, 8, 4, rng)
    ctx = N.Context(0)
    a = ctx.soup_upload(torch.from_numpy(v0).cuda(), torch.from_numpy(t0).cuda(), 4)
    b = ctx.soup_upload(torch.from_numpy(v1).cuda(), torch.from_numpy(t1).cuda(), 8)
    cams = [I.look_at([0.0, 0.0, 3.0], 32, 32)] * 2
    g, col, _ = N.alloc_outputs(cams, 1, 4, "cuda")
    with pytest.raises(N.DsError) as e:
        ctx.raster_forward_multi([a, b], cams, [1, 2], 1, 0, np.zeros(3, np.float32), g, col)
    assert e.value.code == -1
    with pytest.raises(N.DsError) as e:
        ctx.raster_forward_multi([a, 99], cams, [1, 2], 1, 0, np.zeros(3, np.float32), g, col)
    ctx.close()


def test_server_batches_requests_of_different_soups(N):
    """24 requests alternating over 3 soups, queued while paused, then
    released: the first batch holds several requests (hence several soups),
    and every request's output equals its output alone."""
    import torch
    soups, _ = I.serving_workload(n_soups=3, rate=10.0, duration=0.1)
    srv = N.Server(0, n_streams=2, mem_budget=8 << 30, max_batch=8, reserve_pairs=1 << 21)
    ids = [srv.add_soup(torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.tex).cuda(), sc.grid_n)
           for sc in soups]
    rng = np.random.default_rng(12)
    eyes = I.sphere_eyes(24, 3.0, rng)
    reqs = [(i % 3, I.look_at(eyes[i], *I.SERVE_RESOLUTIONS[i % 2]), 1000 + i) for i in range(24)]
    bg = np.zeros(7, np.float32)

    def outputs(cam):
        g = torch.full((1, cam.height, cam.width, 4), -7, dtype=torch.int32, device="cuda")
        col = torch.full((1, 7, cam.height, cam.width), float("nan"), device="cuda")
        return g, col

    alone = []
    for k, cam, seed in reqs:
        g, col = outputs(cam)
        st = srv.wait(srv.submit(ids[k], cam, seed, N.DS_MODE_STOCHASTIC, bg, g, col), 60_000)
        assert st["batch"] == 1
        alone.append((g.cpu(), col.cpu()))
    srv.pause(True)
    outs, tickets = [], []
    for k, cam, seed in reqs:
        g, col = outputs(cam)
        outs.append((g, col))
        tickets.append(srv.submit(ids[k], cam, seed, N.DS_MODE_STOCHASTIC, bg, g, col))
    srv.pause(False)
    stats = [srv.wait(t, 60_000) for t in tickets]
    assert stats[0]["batch"] >= 3          # the oldest request and the next ones, over all three soups
    for i, ((g, col), (ga, ca)) in enumerate(zip(outs, alone)):
        assert torch.equal(g.cpu(), ga), i
        assert torch.equal(col.cpu().view(torch.int32), ca.view(torch.int32)), i
    srv.close()
