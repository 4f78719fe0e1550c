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


def _busy_scene():
    """More tiles (2 x 1280x720: 7,200 tiles of 16x16) and more bin pairs than
    the parity scenes, inside the entry point's limits."""
    rng = np.random.default_rng(60)
    T = 2000
    verts = I.box_soup(T, 0.5, rng)
    tex = I.logits(T, 8, 8, rng)
    cams = [I.look_at(e, 1280, 720) for e in I.sphere_eyes(2, 3.0, rng)]
    return verts, tex, cams


def _render_noalloc(N, verts, tex, grid_n, cams, seeds, S, mode, bg, C):
    import torch
    out = _outputs(N, cams, S, C)
    N.raster_forward_noalloc(torch.from_numpy(verts).cuda(), torch.from_numpy(tex).cuda(), grid_n, cams, seeds, S,
                             mode, bg, *out)
    return out


@pytest.mark.parametrize("scene,S,mode", [("plain", 1, 0), ("plain", 5, 0), ("batched", 1, 0), ("batched", 2, 1)])
def test_noalloc_forward_matches_the_allocating_forward(N, scene, S, mode):
    """Two calls on the same scene, with a call on a larger scene (more tiles,
    more bin pairs) between them: the second call must not see what the
    larger one left in the shared scratch."""
    import torch
    sc = I.plain_small(soup_seed=7, mask_seed=8) if scene == "plain" else I.batched_views()
    verts = torch.from_numpy(sc.verts).cuda()
    tex = torch.from_numpy(sc.tex).cuda()
    ctx = N.Context(0)
    sid = ctx.soup_upload(verts, tex, sc.grid_n)
    ref = _outputs(N, sc.cams, S, sc.C)
    ctx.raster_forward(sid, sc.cams, sc.seeds, S, mode, sc.bg, *ref)
    bv, bt, bc = _busy_scene()
    for call in range(2):                       # two calls on this scene share the scratch
        got = _outputs(N, sc.cams, S, sc.C)
        for t in got[0]:
            t.fill_(-7)                         # stale values must be overwritten
        N.raster_forward_noalloc(verts, tex, sc.grid_n, sc.cams, sc.seeds, S, mode, sc.bg, *got)
        torch.cuda.synchronize()
        _compare(N, got, ref)
        if call == 0:                           # a larger scene in between
            _render_noalloc(N, bv, bt, 8, bc, [91, 92], 3, 0, np.zeros(7, np.float32), 8)
            torch.cuda.synchronize()
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


def test_noalloc_forward_reports_bins_beyond_its_capacity(N):
    """2,000 triangles of edge 1.5 at 1920x1080 pass the up-front limits but
    bin into about 0.9 M (tile, triangle) pairs, beyond the 524,288 the
    scratch holds: DS_ERR_CAPACITY, read back before anything is written
    past the pairs' buffers; a later call still matches the allocating path."""
    import torch
    rng = np.random.default_rng(50)
    T = 2000
    verts, tex = I.box_soup(T, 1.5, rng), I.logits(T, 8, 8, rng)
    cams = [I.look_at([0.0, 0.0, 3.0], 1920, 1080)]
    with pytest.raises(N.DsError) as e:
        _render_noalloc(N, verts, tex, 8, cams, [5], 1, 0, np.zeros(7, np.float32), 8)
    assert e.value.code == -4 and "no-alloc limit" in str(e.value)
    sc = I.plain_small(soup_seed=3, mask_seed=4)
    ctx = N.Context(0)
    v, t = torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.tex).cuda()
    ref = _outputs(N, sc.cams, 2, sc.C)
    ctx.raster_forward(ctx.soup_upload(v, t, sc.grid_n), sc.cams, sc.seeds, 2, 0, sc.bg, *ref)
    got = _render_noalloc(N, sc.verts, sc.tex, sc.grid_n, sc.cams, sc.seeds, 2, 0, sc.bg, sc.C)
    torch.cuda.synchronize()
    _compare(N, got, ref)
    ctx.close()


def test_noalloc_forward_rejects_host_and_misshapen_buffers(N):
    """The binding refuses host tensors and wrong shapes before the call; the
    library itself refuses a host pointer (cudaPointerGetAttributes)."""
    import ctypes
    import torch
    sc = I.plain_small()
    verts, tex = torch.from_numpy(sc.verts), torch.from_numpy(sc.tex)
    g, col, nf = _outputs(N, sc.cams, 1, sc.C)
    with pytest.raises(ValueError):
        N.raster_forward_noalloc(verts, tex.cuda(), sc.grid_n, sc.cams, sc.seeds, 1, 0, sc.bg, g, col, nf)
    with pytest.raises(ValueError):
        N.raster_forward_noalloc(verts.cuda(), tex.cuda(), sc.grid_n + 1, sc.cams, sc.seeds, 1, 0, sc.bg, g, col, nf)
    with pytest.raises(ValueError):
        N.raster_forward_noalloc(verts.cuda(), tex.cuda(), sc.grid_n, sc.cams, sc.seeds, 2, 0, sc.bg, g, col, nf)
    # straight through the C ABI with a host vertex array
    outs = (N.ds_view_out * 1)()
    outs[0].gbuf, outs[0].color, outs[0].n_front = g[0].data_ptr(), col[0].data_ptr(), None
    T, V, C = sc.tex.shape
    vh = np.ascontiguousarray(sc.verts)
    bg = np.ascontiguousarray(sc.bg, np.float32)
    seeds = (ctypes.c_uint64 * 1)(int(sc.seeds[0]))
    td = tex.cuda()
    rc = N.load().ds_raster_forward_noalloc(vh.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(td.data_ptr()),
                                            T, sc.grid_n, C, N.cameras(sc.cams), seeds, 1, 1, 0,
                                            bg.ctypes.data_as(ctypes.c_void_p), outs,
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1 and "device memory" in N.load().ds_last_error().decode()
