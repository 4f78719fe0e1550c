"""Pins of the L1 + SSIM oracle (oracle/ssim.py): identity and symmetry,
the constant-image closed form away from the border, the window, and the
gradient against central differences of sum_p ell_p."""
import numpy as np

from oracle import ssim as SS


def test_identity_and_symmetry():
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, (3, 20, 17))
    y = rng.uniform(0, 1, (3, 20, 17))
    assert np.allclose(SS.ssim_map(x, x), 1.0, atol=1e-12)
    ell, g = SS.loss(x[None], x)
    assert np.allclose(ell, 0.0, atol=1e-12)
    assert np.allclose(SS.ssim_map(x, y), SS.ssim_map(y, x), atol=1e-14)


def test_constant_images_closed_form():
    a, b = 0.3, 0.7
    s = SS.ssim_map(np.full((1, 30, 30), a), np.full((1, 30, 30), b))
    inner = s[0, 5:25, 5:25]                   # the window lies inside the image
    assert np.allclose(inner, (2 * a * b + SS.C1) / (a * a + b * b + SS.C1), rtol=1e-12)
    ell, _ = SS.loss(np.full((1, 1, 30, 30), a), np.full((1, 30, 30), b), lam=0.8)
    assert np.allclose(ell[0, 5:25, 5:25], 0.8 * abs(a - b) + 0.2 * (1 - inner), rtol=1e-12)


def test_window():
    w = SS.window1d()
    assert np.isclose(w.sum(), 1.0) and np.allclose(w, w[::-1]) and len(w) == 11
    img = np.zeros((1, 21, 21)); img[0, 10, 10] = 1.0
    assert np.allclose(SS.blur(img)[0, 5:16, 5:16], np.outer(w, w))   # impulse response = the 2D window


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    x = rng.uniform(0.05, 0.95, (2, 3, 14, 12))
    y = rng.uniform(0, 1, (3, 14, 12))
    _, g = SS.loss(x, y)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (1, 2, 7, 5), (0, 1, 13, 11), (1, 0, 3, 9), (0, 2, 6, 0)]:
        e = np.zeros_like(x); e[idx] = h
        fd = (SS.loss(x + e, y)[0].sum() - SS.loss(x - e, y)[0].sum()) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, g[idx])
