"""The deferred-shading forward on the tensor cores (tcgen05 MMAs of
kind::tf32 with every operand split into a TF32 high part and the
remainder) against the FP64 oracle (oracle/shading.py) and against the
CUDA-core kernel, on the same seeded inputs.

Tolerance: rgb within 1e-5 of the oracle, as for the CUDA-core kernel (the
split keeps about 21 bits of every product; the dropped lo x lo term and the
tensor cores' FP32 accumulation order leave a few 1e-7)."""
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
    return SH.pack(W1, rng.normal(0, 0.3, 16), W2, rng.normal(0, 0.3, 16), W3, rng.normal(0, 0.3, 3))


def _to(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _shade(ctx, path, cams, params, feats):
    import torch
    from paper_2603_27151_gb300 import native as N
    path0 = ctx.get_shade_path()
    ctx.set_shade_path(path)
    f = [_to(x) for x in feats]
    rgb = [torch.full((x.shape[0], 3, x.shape[2], x.shape[3]), -1.0, device="cuda") for x in feats]
    ctx.shade_forward(cams, _to(params.astype(np.float32)), f, rgb)
    torch.cuda.synchronize()
    ctx.set_shade_path(path0)
    ctx.status()                                   # no timed-out MMA wait
    return [r.cpu().numpy() for r in rgb]


@pytest.mark.parametrize("S", [1, 3, 4])
def test_tensor_core_forward_matches_the_oracle_and_the_cuda_cores(ctx, S):
    """Three views (96x64, 37x23, 300x17): tiles of 128 pixels, each taking
    all S samples, with ragged ends in every view."""
    from paper_2603_27151_gb300 import native as N
    eyes = I.sphere_eyes(3, 3.0, np.random.default_rng(4))
    cams = [I.look_at(eyes[0], 96, 64), I.look_at(eyes[1], 37, 23), I.look_at(eyes[2], 300, 17)]
    rng = np.random.default_rng(2)
    feats = [rng.uniform(0, 1, (S, 7, c.height, c.width)).astype(np.float32) for c in cams]
    params = _params()
    tc = _shade(ctx, N.DS_SHADE_TENSOR_CORES, cams, params, feats)
    cc = _shade(ctx, N.DS_SHADE_CUDA_CORES, cams, params, feats)
    for v, c in enumerate(cams):
        ref = SH.shade(feats[v], c, params)
        assert np.abs(tc[v] - ref).max() <= 1e-5, (v, float(np.abs(tc[v] - ref).max()))
        assert np.abs(cc[v] - ref).max() <= 1e-5, (v, float(np.abs(cc[v] - ref).max()))
        assert np.abs(tc[v] - cc[v]).max() <= 1e-5, v


def test_tensor_core_forward_tiny_views(ctx):
    """Views smaller than one tile of 128 pixels (1x1, 5x3) beside a normal
    one: every tile partial, S = 2."""
    from paper_2603_27151_gb300 import native as N
    eyes = I.sphere_eyes(3, 3.0, np.random.default_rng(6))
    cams = [I.look_at(eyes[0], 1, 1), I.look_at(eyes[1], 5, 3), I.look_at(eyes[2], 40, 20)]
    rng = np.random.default_rng(3)
    feats = [rng.uniform(0, 1, (2, 7, c.height, c.width)).astype(np.float32) for c in cams]
    params = _params(17)
    tc = _shade(ctx, N.DS_SHADE_TENSOR_CORES, cams, params, feats)
    for v, c in enumerate(cams):
        ref = SH.shade(feats[v], c, params)
        assert np.abs(tc[v] - ref).max() <= 1e-5, v


def test_tensor_core_forward_special_cases(ctx):
    """A = 1 returns the feature colour exactly; all-zero features give the
    MLP of the view direction alone; large weights and biases (ReLU on both
    sides, saturating outputs) stay within tolerance."""
    from paper_2603_27151_gb300 import native as N
    cams = [I.look_at([0.0, -3.0, 0.5], 64, 32), I.look_at([2.0, 2.0, 1.0], 33, 20)]
    rng = np.random.default_rng(9)
    feats = [rng.uniform(0, 1, (2, 7, c.height, c.width)).astype(np.float32) for c in cams]
    feats[0][:, 3] = 1.0
    feats[1][:] = 0.0
    params = _params(5) * np.float32(3.0)
    tc = _shade(ctx, N.DS_SHADE_TENSOR_CORES, cams, params, feats)
    assert np.array_equal(tc[0], feats[0][:, 0:3])
    for v, c in enumerate(cams):
        ref = SH.shade(feats[v], c, params)
        assert np.abs(tc[v] - ref).max() <= 1e-5, v


def test_shade_path_setting(ctx):
    """A new context shades on the tensor cores; the setting persists and
    rejects unknown paths."""
    from paper_2603_27151_gb300 import native as N
    fresh = N.Context(0)
    try:
        assert fresh.get_shade_path() == N.DS_SHADE_TENSOR_CORES
    finally:
        fresh.close()
    path0 = ctx.get_shade_path()
    ctx.set_shade_path(N.DS_SHADE_CUDA_CORES)
    assert ctx.get_shade_path() == N.DS_SHADE_CUDA_CORES
    with pytest.raises(N.DsError):
        ctx.set_shade_path(7)
    assert ctx.get_shade_path() == N.DS_SHADE_CUDA_CORES
    ctx.set_shade_path(N.DS_SHADE_TENSOR_CORES)
    assert ctx.get_shade_path() == N.DS_SHADE_TENSOR_CORES
    ctx.set_shade_path(path0)


def test_tensor_core_wait_runs_out_and_the_context_recovers(ctx):
    """The bounded wait of the tensor-core kernel on the GPU: with the MMAs
    never issued, every CTA's wait for them runs out (about 2 s), the CTA
    releases its tensor memory and returns without writing, the status check
    reports DS_ERR_TIMEOUT once, and the same context then shades correctly."""
    import torch
    from paper_2603_27151_gb300 import native as N
    cams = [I.look_at([0.0, -3.0, 0.5], 64, 32)]
    rng = np.random.default_rng(12)
    feats = [rng.uniform(0, 1, (2, 7, 32, 64)).astype(np.float32)]
    params = _params(13)
    path0 = ctx.get_shade_path()
    ctx.set_shade_path(N.DS_SHADE_TENSOR_CORES_WAIT_TEST)
    assert ctx.get_shade_path() == N.DS_SHADE_TENSOR_CORES_WAIT_TEST
    rgb = [torch.full((2, 3, 32, 64), -1.0, device="cuda")]
    ctx.shade_forward(cams, _to(params.astype(np.float32)), [_to(feats[0])], rgb)
    torch.cuda.synchronize()
    ctx.set_shade_path(path0)
    with pytest.raises(N.DsError) as e:
        ctx.status()
    assert e.value.code == -5                      # DS_ERR_TIMEOUT
    assert bool((rgb[0] == -1.0).all())            # nothing written
    ctx.status()                                   # reported once
    got = _shade(ctx, N.DS_SHADE_TENSOR_CORES, cams, params, feats)
    assert np.abs(got[0] - SH.shade(feats[0], cams[0], params)).max() <= 1e-5


def test_tensor_core_forward_full_size_batch(ctx):
    """The 1080p batch's colour features (4 x 1920x1080 + 4 x 960x540, S = 4,
    41.5 M pixel-samples, 81,000 tiles of 128 pixels) in one launch: windows at corners
    and the centre against the oracle on cropped cameras, everything against
    the CUDA-core kernel."""
    import torch
    from paper_2603_27151_gb300 import native as N
    sc = I.large_batch()
    S = sc.samples
    sid = ctx.soup_upload(_to(sc.verts), _to(sc.tex), sc.grid_n)
    g, col, _ = N.alloc_outputs(sc.cams, S, sc.C, "cuda", n_front=False)
    ctx.raster_forward(sid, sc.cams, sc.seeds, S, 0, sc.bg, g, col)
    params = _params(21)
    p = _to(params.astype(np.float32))
    out = {}
    for path in (N.DS_SHADE_TENSOR_CORES, N.DS_SHADE_CUDA_CORES):
        ctx.set_shade_path(path)
        rgb = [torch.empty((S, 3, c.height, c.width), device="cuda") for c in sc.cams]
        ctx.shade_forward(sc.cams, p, col, rgb)
        torch.cuda.synchronize()
        out[path] = rgb
    ctx.set_shade_path(N.DS_SHADE_TENSOR_CORES)
    ctx.status()
    for v, c in enumerate(sc.cams):
        d = (out[N.DS_SHADE_TENSOR_CORES][v] - out[N.DS_SHADE_CUDA_CORES][v]).abs().max().item()
        assert d <= 1e-5, (v, d)
        for (x0, y0) in [(0, 0), (c.width - 40, c.height - 24), (c.width // 2 - 13, c.height // 3)]:
            w, h = 40, 24
            cam = I.Camera(w, h, c.fx, c.fy, c.cx - x0, c.cy - y0, c.R, c.t, c.near)
            fwin = col[v][:, :, y0:y0 + h, x0:x0 + w].cpu().numpy()
            ref = SH.shade(fwin, cam, params)
            got = out[N.DS_SHADE_TENSOR_CORES][v][:, :, y0:y0 + h, x0:x0 + w].cpu().numpy()
            assert np.abs(got - ref).max() <= 1e-5, (v, x0, y0)
    ctx.soup_free(sid)
