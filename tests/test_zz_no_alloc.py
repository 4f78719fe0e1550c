"""ds_raster_forward_noalloc: the forward pass for callers that cannot
allocate device memory (engines that own all device memory through their own
pool, programs under a hard memory budget, real-time loops that cannot take
cudaMalloc's synchronisation).  Its scratch is a fixed array inside the
library.  It must give the same outputs as ds_raster_forward, call after call:
the array keeps the previous call's contents, so a second call in a row checks
that everything that must start at zero is cleared.  This file is collected
last so that a run that stops at the first failure has run every other test;
it also passes on its own in a fresh process."""
import numpy as np
import pytest

from paper_2603_27151_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_27151_gb300 import native
    return native


def _outputs(N, cams, S, C):
    return N.alloc_outputs(cams, S, C, "cuda", n_front=True)


def _compare(N, a, b):
    (ga, ca, fa), (gb, cb, fb) = a, b
    for v in range(len(ga)):
        ta, ba, da = N.split_gbuf(ga[v])
        tb, bb, db = N.split_gbuf(gb[v])
        assert np.array_equal(ta.cpu().numpy(), tb.cpu().numpy())
        assert np.array_equal(ba.cpu().numpy(), bb.cpu().numpy())
        assert np.array_equal(da.cpu().numpy(), db.cpu().numpy())
        assert np.array_equal(fa[v].cpu().numpy(), fb[v].cpu().numpy())
        x, y = ca[v].cpu().numpy(), cb[v].cpu().numpy()
        assert np.all(np.abs(x - y) <= 1e-5 * np.abs(y) + 1e-7)


@pytest.mark.parametrize("scene,S,mode", [("plain", 1, 0), ("plain", 5, 0), ("batched", 1, 0), ("batched", 2, 1)])
def test_noalloc_forward_matches_the_allocating_forward(N, scene, S, mode):
    import torch
    sc = I.plain_small(soup_seed=7, mask_seed=8) if scene == "plain" else I.batched_views()
    verts = torch.from_numpy(sc.verts).cuda()
    tex = torch.from_numpy(sc.tex).cuda()
    ctx = N.Context(0)
    sid = ctx.soup_upload(verts, tex, sc.grid_n)
    ref = _outputs(N, sc.cams, S, sc.C)
    ctx.raster_forward(sid, sc.cams, sc.seeds, S, mode, sc.bg, *ref)
    for call in range(2):                       # two calls in a row share the scratch
        got = _outputs(N, sc.cams, S, sc.C)
        for t in got[0]:
            t.fill_(-7)                         # stale values must be overwritten
        N.raster_forward_noalloc(verts, tex, sc.grid_n, sc.cams, sc.seeds, S, mode, sc.bg, *got)
        torch.cuda.synchronize()
        _compare(N, got, ref)
    ctx.close()


def test_noalloc_forward_rejects_sizes_beyond_its_limit(N):
    import torch
    sc = I.large_batch()                        # 100,000 triangles x 45 texels x 8 channels
    verts = torch.from_numpy(sc.verts[:20000]).cuda()
    tex = torch.from_numpy(sc.tex[:20000]).cuda()
    g, col, nf = _outputs(N, sc.cams[:1], 1, sc.C)
    with pytest.raises(N.DsError) as e:
        N.raster_forward_noalloc(verts, tex, sc.grid_n, sc.cams[:1], sc.seeds[:1], 1, 0, sc.bg, g, col, nf)
    assert e.value.code == -1 and "no-alloc limit" in str(e.value)
