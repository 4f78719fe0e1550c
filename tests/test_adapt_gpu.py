"""GPU parity of the adaptive control of primitives (Sec. 3.4) against the
oracle on the same seeded inputs: coverage counts, edge ratios (FP32 in the
oracle's order: the same bits, since they decide the splits), the rebuilt
soup (bit for bit) and one whole round."""
import numpy as np
import pytest

import oracle as O
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


def _views(n, seed, res=(160, 120)):
    eyes = I.sphere_eyes(n, 3.0, np.random.default_rng(seed))
    return [I.look_at(e, res[0], res[1]) for e in eyes]


def test_coverage_counts(ctx):
    import torch
    from paper_2603_27151_gb300 import native as N
    sc = I.batched_views()
    S = 3
    ref = O.forward(sc.verts, sc.tex, sc.grid_n, sc.cams, sc.seeds, S=S, bg=sc.bg)
    want = O.coverage([r["tri_id"] for r in ref], sc.T)
    sid = ctx.soup_upload(torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.tex).cuda(), sc.grid_n)
    g, col, _ = N.alloc_outputs(sc.cams, S, sc.C, "cuda")
    ctx.raster_forward(sid, sc.cams, sc.seeds, S, 0, sc.bg, g, col)
    counts = torch.zeros(sc.T, dtype=torch.int32, device="cuda")
    N.coverage_count(g, sc.T, counts)
    torch.cuda.synchronize()
    assert np.array_equal(counts.cpu().numpy().astype(np.int64), want)
    N.coverage_count(g[:2], sc.T, counts)      # accumulates
    torch.cuda.synchronize()
    assert np.array_equal(counts.cpu().numpy().astype(np.int64),
                          want + O.coverage([r["tri_id"] for r in ref[:2]], sc.T))
    ctx.soup_free(sid)


def test_edge_ratios_bit_exact(ctx):
    import torch
    from paper_2603_27151_gb300 import native as N
    sc = I.batched_views()
    cams = _views(20, 31, (640, 480)) + [I.look_at([0.2, 0.1, 0.5], 320, 240)]   # one view inside the soup
    out = torch.empty((sc.T, 3), device="cuda")
    N.edge_ratios(torch.from_numpy(sc.verts).cuda(), cams, out)
    torch.cuda.synchronize()
    want = O.edge_ratios(sc.verts, cams)
    assert np.array_equal(out.cpu().numpy(), want)
    assert (want > 0.2).any() and (want < 0.2).any()


@pytest.mark.parametrize("levels", [(3, 3), (1, 4)])
def test_rebuild_bit_exact(ctx, levels):
    import torch
    from paper_2603_27151_gb300 import native as N
    r_min, r_max = levels
    T, C = 300, 8
    rng = np.random.default_rng(9)
    verts = I.box_soup(T, 0.3, rng)
    lv = I.level_logits(T, r_min, r_max, C, rng)
    counts = rng.integers(0, 40, size=T)
    ratios = rng.uniform(0, 0.4, size=(T, 3)).astype(np.float32)
    plan = O.adapt_plan(counts, ratios, 0.2, 340)
    vo_ref, lo_ref = O.soup_rebuild(verts, lv, r_min, r_max, plan)
    n = len(plan)
    tex = torch.from_numpy(np.concatenate([l.reshape(-1) for l in lv])).cuda()
    vo = torch.empty((n, 3, 3), device="cuda")
    to = torch.empty(sum(N.level_sizes(n, r_min, r_max, C)), device="cuda")
    ctx.soup_rebuild(torch.from_numpy(verts).cuda(), tex, T, [1 << R for R in range(r_min, r_max + 1)], C,
                     N.adapt_plan(counts, ratios, 0.2, 340), vo, to)
    assert np.array_equal(vo.cpu().numpy(), vo_ref)
    for a, b in zip(N.split_levels(to, n, r_min, r_max, C), lo_ref):
        assert np.array_equal(a.cpu().numpy(), b)


def test_rebuild_rejects_a_bad_plan(ctx):
    import torch
    from paper_2603_27151_gb300 import native as N
    v = torch.zeros((4, 3, 3), device="cuda")
    t = torch.zeros((4, 15, 2), device="cuda")
    for bad in ([4 << 3], [0 << 3 | 7], [-8]):
        with pytest.raises(N.DsError):
            ctx.soup_rebuild(v, t, 4, [4], 2, np.array(bad, np.int32), torch.empty((1, 3, 3), device="cuda"),
                             torch.empty((1, 15, 2), device="cuda"))


def test_one_round_matches_the_oracle(ctx):
    """Render the training views, count coverage, measure edges on 20 views,
    plan with a budget, rebuild: the new soup is the oracle's, bit for bit."""
    import torch
    from paper_2603_27151_gb300 import native as N
    rng = np.random.default_rng(17)
    T, r_min, r_max, C = 600, 1, 3, 8
    verts = I.box_soup(T, 0.25, rng)
    lv = I.level_logits(T, r_min, r_max, C, rng)
    train = _views(6, 41, (128, 96))
    measure = _views(20, 43, (256, 192))
    bg = np.zeros(C - 1, np.float32)
    # oracle round
    ref = O.forward_levels(verts, lv, r_min, r_max, train, None, S=1, mode=O.MODE_THRESHOLD_HALF, bg=bg)
    counts = O.coverage([r["tri_id"] for r in ref], T)
    ratios = O.edge_ratios(verts, measure)
    plan = O.adapt_plan(counts, ratios, 0.15, 700)
    v_ref, l_ref = O.soup_rebuild(verts, lv, r_min, r_max, plan)
    # library round
    vt = torch.from_numpy(verts).cuda()
    tt = torch.from_numpy(np.concatenate([l.reshape(-1) for l in lv])).cuda()
    sid = ctx.soup_upload_levels(vt, tt, T, r_min, r_max, C)
    g, col, _ = N.alloc_outputs(train, 1, C, "cuda")
    ctx.raster_forward(sid, train, None, 1, N.DS_MODE_THRESHOLD_HALF, bg, g, col)
    cnt = torch.zeros(T, dtype=torch.int32, device="cuda")
    N.coverage_count(g, T, cnt)
    rat = torch.empty((T, 3), device="cuda")
    N.edge_ratios(vt, measure, rat)
    torch.cuda.synchronize()
    pl = N.adapt_plan(cnt.cpu().numpy(), rat.cpu().numpy(), 0.15, 700)
    assert np.array_equal(pl, plan)
    n = len(pl)
    vo = torch.empty((n, 3, 3), device="cuda")
    to = torch.empty(sum(N.level_sizes(n, r_min, r_max, C)), device="cuda")
    ctx.soup_rebuild(vt, tt, T, [1 << R for R in range(r_min, r_max + 1)], C, pl, vo, to)
    assert np.array_equal(vo.cpu().numpy(), v_ref)
    for a, b in zip(N.split_levels(to, n, r_min, r_max, C), l_ref):
        assert np.array_equal(a.cpu().numpy(), b)
    assert 699 <= n <= 700 and (pl & 7).any() and len(set((pl >> 3).tolist())) < T   # split and pruned
    ctx.soup_free(sid)
