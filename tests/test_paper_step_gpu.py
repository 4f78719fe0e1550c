"""The full training step of the paper through the library (level soup ->
stochastic forward -> deferred shading -> L1 + SSIM -> shading backward ->
rasteriser backward -> VectorAdam / Adam), against the same chain of CPU
oracles on the same seeded inputs: visibility bit for bit, RGB within 1e-5,
the loss within 1e-4 relative and every gradient within 1e-3 (the FP32
differences of the shading and SSIM stages propagate into the backward's
upstream values); and the loss decreases over a few steps."""
import numpy as np
import pytest

import oracle as O
from oracle import shading as SH
from oracle import ssim as SS
from paper_2603_27151_gb300 import inputs as I
from tests.gpu_helpers import grad_mismatch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return "cuda"


def _scene(seed=31, T=400, r_min=1, r_max=3, n_views=3, res=(64, 48)):
    rng = np.random.default_rng(seed)
    verts = I.box_soup(T, 0.3, rng)
    lv = I.level_logits(T, r_min, r_max, 8, rng)
    eyes = I.sphere_eyes(n_views, 3.0, np.random.default_rng(seed + 1))
    cams = [I.look_at(e, res[0], res[1]) for e in eyes]
    targets = [rng.uniform(0, 1, (3, res[1], res[0])).astype(np.float32) for _ in cams]
    W1, b1, W2, b2, W3, b3 = SH.unpack(SH.xavier_params(seed))
    params = SH.pack(W1, rng.normal(0, 0.2, 16), W2, rng.normal(0, 0.2, 16), W3, rng.normal(0, 0.2, 3))
    return verts, lv, cams, targets, params.astype(np.float32)


def test_paper_step_matches_the_oracle_chain(dev):
    import torch
    from paper_2603_27151_gb300.paper_step import PaperStep
    r_min, r_max, S = 1, 3, 2
    verts, lv, cams, targets, params = _scene()
    T = verts.shape[0]
    vt = torch.from_numpy(verts).cuda()
    tt = torch.from_numpy(np.concatenate([l.reshape(-1) for l in lv])).cuda()
    st = PaperStep(vt, tt, T, r_min, r_max, 8, cams, [torch.from_numpy(t).cuda() for t in targets], S=S,
                   params=torch.from_numpy(params).cuda())
    ids = [0, 2]
    seeds = I.mask_seeds(7, len(ids))
    rgb = st.gradients(ids, seeds)
    torch.cuda.synchronize()
    # the oracle chain
    vcams = [cams[k] for k in ids]
    p64 = params.astype(np.float64)
    ref = O.forward_levels(verts, lv, r_min, r_max, vcams, seeds, S=S, bg=np.zeros(7, np.float32))
    gcol, sws, gp_ref, loss_ref = [], [], np.zeros(SH.N_PARAMS), 0.0
    for v, (k, cam) in enumerate(zip(ids, vcams)):
        feat = ref[v]["color"].astype(np.float64)
        rgb_ref = SH.shade(feat, cam, p64)
        assert np.abs(rgb[v].cpu().numpy() - rgb_ref).max() <= 1e-5
        ell, g_rgb = SS.loss(rgb_ref, targets[k].astype(np.float64))
        gf, gp = SH.shade_backward(feat, cam, p64, g_rgb / S)
        gcol.append(gf.astype(np.float32))
        sws.append((ell / S).astype(np.float32))
        gp_ref += gp
        loss_ref += float(ell.sum()) / S
    gl_ref, gv_ref = O.backward_levels(verts, lv, r_min, r_max, vcams, S, ref, gcol, sws)
    assert abs(float(st.loss) - loss_ref) <= 1e-4 * loss_ref
    gp = st.g_params.cpu().numpy()
    assert np.all(np.abs(gp - gp_ref) <= 1e-3 * (np.abs(gp_ref) + 1e-2 * np.abs(gp_ref).max()))
    from paper_2603_27151_gb300 import native as N
    for R, a, b in zip(range(r_min, r_max + 1), N.split_levels(st.g_tex, T, r_min, r_max, 8), gl_ref):
        bad = grad_mismatch(a.cpu().numpy(), b, rtol=1e-3)
        assert not bad.any(), "level %d: %d of %d" % (R, bad.sum(), bad.size)
    assert grad_mismatch(st.g_verts.cpu().numpy(), gv_ref, rtol=1e-3).mean() < 1e-3
    st.close()


def test_paper_step_decreases_the_loss(dev):
    import torch
    from paper_2603_27151_gb300.paper_step import PaperStep
    verts, lv, cams, targets, params = _scene(seed=5, n_views=4)
    T = verts.shape[0]
    vt = torch.from_numpy(verts).cuda()
    tt = torch.from_numpy(np.concatenate([l.reshape(-1) for l in lv])).cuda()
    st = PaperStep(vt, tt, T, 1, 3, 8, cams, [torch.from_numpy(t).cuda() for t in targets], S=1, per_step=4,
                   total_steps=60, params=torch.from_numpy(params).cuda())
    losses = [st.step() for _ in range(40)]
    assert np.all(np.isfinite(losses))
    assert np.mean(losses[-5:]) < 0.9 * np.mean(losses[:5]), (losses[:5], losses[-5:])
    assert torch.isfinite(vt).all() and torch.isfinite(tt).all() and torch.isfinite(st.params).all()
    st.close()
