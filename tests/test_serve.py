"""Render server (continuous batching over resident soups).

A request's pixels depend only on its soup, camera and seed, so its output
must be bit-identical whether it runs alone, batched with other requests
(mixed soups, modes and resolutions), or through a direct forward call; on a
small case it must equal the oracle.  Admission by memory budget, pause,
time-outs and the error paths are checked as well."""
import numpy as np
import pytest

import oracle as O
from paper_2603_27151_gb300 import inputs as I
from tests.gpu_helpers import assert_forward_equal

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


def _outputs(cam, C):
    import torch
    g = torch.empty((1, cam.height, cam.width, 4), dtype=torch.int32, device="cuda")
    col = torch.empty((1, C - 1, cam.height, cam.width), dtype=torch.float32, device="cuda")
    return g, col


def _upload(N, srv, soups):
    import torch
    ids = []
    for sc in soups:
        ids.append(srv.add_soup(torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.tex).cuda(), sc.grid_n))
    return ids


def _mode(i, N):
    return N.DS_MODE_THRESHOLD_HALF if i % 3 == 0 else N.DS_MODE_STOCHASTIC


def test_alone_equals_mixed_and_direct(lib):
    import torch
    N = lib
    soups, reqs = I.serving_workload(n_soups=3, rate=300.0, duration=0.1)
    assert len(reqs) >= 20
    srv = N.Server(0, n_streams=3, mem_budget=8 << 30, max_batch=8, reserve_pairs=1 << 21)
    ids = _upload(N, srv, soups)
    bg = np.zeros(7, np.float32)
    alone = []
    for i, (_, k, cam, seed) in enumerate(reqs):
        g, col = _outputs(cam, 8)
        st = srv.wait(srv.submit(ids[k], cam, seed, _mode(i, N), bg, g, col))
        assert st["batch"] == 1
        alone.append((g.cpu(), col.cpu()))
    # the same requests queued at once (paused), then released: they batch
    srv.pause(True)
    outs, tickets = [], []
    for i, (_, k, cam, seed) in enumerate(reqs):
        g, col = _outputs(cam, 8)
        g.fill_(-7)
        col.fill_(float("nan"))
        outs.append((g, col))
        tickets.append(srv.submit(ids[k], cam, seed, _mode(i, N), bg, g, col))
    srv.pause(False)
    stats = [srv.wait(t, 60_000) for t in tickets]
    assert max(s["batch"] for s in stats) > 1
    for i, ((g, col), (ga, ca)) in enumerate(zip(outs, alone)):
        assert torch.equal(g.cpu(), ga), "request %d: G-buffer differs between alone and batched" % i
        assert torch.equal(col.cpu().view(torch.int32), ca.view(torch.int32)), "request %d: colour differs" % i
    # a direct forward call gives the same bits
    ctx = N.Context(0)
    for i in range(0, len(reqs), 5):
        _, k, cam, seed = reqs[i]
        sid = ctx.soup_upload(torch.from_numpy(soups[k].verts).cuda(), torch.from_numpy(soups[k].tex).cuda(), 8)
        g, col = _outputs(cam, 8)
        ctx.raster_forward(sid, [cam], [seed], 1, _mode(i, N), bg, [g], [col])
        torch.cuda.synchronize()
        assert torch.equal(g.cpu(), alone[i][0])
        assert torch.equal(col.cpu().view(torch.int32), alone[i][1].view(torch.int32))
        ctx.soup_free(sid)
    ctx.close()
    srv.close()


def test_server_matches_oracle(lib):
    import torch
    N = lib
    sc = I.plain_small()
    srv = N.Server(0, n_streams=2, mem_budget=1 << 28, max_batch=4, reserve_pairs=1 << 16)
    (sid,) = _upload(N, srv, [sc])
    cam, seed = sc.cams[0], int(sc.seeds[0])
    g, col = _outputs(cam, sc.C)
    srv.wait(srv.submit(sid, cam, seed, N.DS_MODE_STOCHASTIC, sc.bg, g, col), 60_000)
    tri, bary, depth = N.split_gbuf(g)
    got = [dict(tri_id=tri.cpu().numpy(), bary=bary.cpu().numpy(), depth=depth.cpu().numpy(),
                color=col.cpu().numpy(), n_front=None)]
    ref = O.forward(sc.verts, sc.tex, sc.grid_n, [cam], [seed], S=1, mode=O.MODE_STOCHASTIC, bg=sc.bg)
    assert_forward_equal(got, ref)
    srv.close()


def test_memory_budget_serialises(lib):
    """With a budget below one request, batches hold one request each and run
    one at a time (each launch after the previous completion)."""
    N = lib
    soups, reqs = I.serving_workload(n_soups=2, rate=200.0, duration=0.05)
    srv = N.Server(0, n_streams=3, mem_budget=1, max_batch=8, reserve_pairs=1 << 21)
    ids = _upload(N, srv, soups)
    srv.pause(True)
    keep, tickets = [], []
    for i, (_, k, cam, seed) in enumerate(reqs):
        g, col = _outputs(cam, 8)
        keep.append((g, col))
        tickets.append(srv.submit(ids[k], cam, seed, N.DS_MODE_STOCHASTIC, None, g, col))
    srv.pause(False)
    stats = sorted((srv.wait(t, 60_000) for t in tickets), key=lambda s: s["launch_ns"])
    assert all(s["batch"] == 1 for s in stats)
    for a, b in zip(stats, stats[1:]):
        assert b["launch_ns"] >= a["done_ns"]
    srv.close()


def test_server_errors(lib):
    import torch
    N = lib
    sc = I.plain_small()
    srv = N.Server(0, n_streams=1, mem_budget=1 << 28, max_batch=4, reserve_pairs=1 << 16)
    (sid,) = _upload(N, srv, [sc])
    cam = sc.cams[0]
    g, col = _outputs(cam, sc.C)
    with pytest.raises(N.DsError) as e:
        srv.submit(sid + 5, cam, 0, N.DS_MODE_STOCHASTIC, sc.bg, g, col)
    assert e.value.code == -6
    bad = I.Camera(**{**cam.__dict__, "width": 0})
    with pytest.raises(N.DsError) as e:
        srv.submit(sid, bad, 0, N.DS_MODE_STOCHASTIC, sc.bg, g, col)
    assert e.value.code == -1
    with pytest.raises(N.DsError) as e:
        srv.wait(123456789, 10)
    assert e.value.code == -6
    # a paused request times out, then completes after resume
    srv.pause(True)
    tk = srv.submit(sid, cam, 0, N.DS_MODE_STOCHASTIC, sc.bg, g, col)
    with pytest.raises(N.DsError) as e:
        srv.wait(tk, 50)
    assert e.value.code == -5
    srv.pause(False)
    srv.wait(tk, 60_000)
    torch.cuda.synchronize()
    # queued requests are cancelled by destroy
    srv.pause(True)
    tk2 = srv.submit(sid, cam, 1, N.DS_MODE_STOCHASTIC, sc.bg, g, col)
    srv.close()
    del tk2
