"""Shared helpers of the GPU parity tests: run the C-ABI path and compare it
with the oracle on identical seeded inputs."""
import numpy as np

import oracle as O
from paper_2603_27151_gb300 import native as N


def gpu_forward(ctx, sc, S=None, mode=0, n_front=True, verts=None, tex=None):
    import torch
    S = S or sc.samples
    verts = torch.from_numpy(sc.verts).cuda() if verts is None else verts
    tex = torch.from_numpy(sc.tex).cuda() if tex is None else tex
    sid = ctx.soup_upload(verts, tex, sc.grid_n)
    g, col, nf = N.alloc_outputs(sc.cams, S, sc.C, "cuda", n_front=n_front)
    ctx.raster_forward(sid, sc.cams, sc.seeds, S, mode, sc.bg, g, col, nf)
    torch.cuda.synchronize()
    out = []
    for v in range(len(sc.cams)):
        tri, bary, depth = N.split_gbuf(g[v])
        out.append(dict(tri_id=tri.cpu().numpy(), bary=bary.cpu().numpy(), depth=depth.cpu().numpy(),
                        color=col[v].cpu().numpy(), n_front=None if nf is None else nf[v].cpu().numpy()))
    return sid, out, (g, col, verts, tex)


def assert_forward_equal(got, ref, views=None, color_rtol=1e-5):
    for v, (a, b) in enumerate(zip(got, ref)):
        if views is not None and v not in views:
            continue
        assert np.array_equal(a["tri_id"], b["tri_id"]), "view %d: tri_id differs at %d pixels" % (
            v, int((a["tri_id"] != b["tri_id"]).sum()))
        if a["n_front"] is not None:
            assert np.array_equal(a["n_front"], b["n_front"]), "view %d: n_front differs" % v
        assert np.array_equal(a["bary"], b["bary"]), "view %d: barycentrics differ" % v
        assert np.array_equal(a["depth"], b["depth"]), "view %d: depth differs" % v
        err = np.abs(a["color"] - b["color"])
        assert np.all(err <= color_rtol * np.abs(b["color"]) + 1e-7), "view %d: colour max err %g" % (v, err.max())


def grad_mismatch(got, want, rtol=1e-4, floor=1e-3):
    """Entries violating |g - ref| <= rtol * max(|ref|, floor * max|ref|)."""
    tol = rtol * np.maximum(np.abs(want), floor * np.abs(want).max())
    return np.abs(got - want) > tol


def upstream(ref_views, S, seed=0):
    """Random upstream gradients and score weights shaped like the outputs."""
    rng = np.random.default_rng(seed)
    gc = [rng.standard_normal(f["color"].shape).astype(np.float32) for f in ref_views]
    sw = [rng.uniform(0.1, 1.0, f["tri_id"].shape).astype(np.float32) for f in ref_views]
    return gc, sw


def gpu_backward(ctx, sid, sc, S, g, col, gc, sw, flags, verts, tex):
    import torch
    gt = torch.zeros_like(tex)
    gv = torch.zeros_like(verts)
    ctx.raster_backward(sid, sc.cams, S, g, col, [torch.from_numpy(x).cuda() for x in gc],
                        [torch.from_numpy(x).cuda() for x in sw], flags, gv, gt)
    torch.cuda.synchronize()
    return gt.cpu().numpy(), gv.cpu().numpy()
