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


def test_ssim_map_against_a_direct_window_sum():
    """At single pixels (corners, edges, interior) the map equals the SSIM
    formula evaluated with an explicit 11x11 Gaussian-weighted sum over the
    zero-padded neighbourhood (no separable passes)."""
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 1, (1, 17, 23))
    y = rng.uniform(0, 1, (1, 17, 23))
    w1 = SS.window1d()
    w2 = np.outer(w1, w1)
    s = SS.ssim_map(x, y)[0]
    for (r, c) in [(0, 0), (16, 22), (0, 11), (8, 0), (8, 11), (3, 19)]:
        m = {k: 0.0 for k in ("x", "y", "xx", "yy", "xy")}
        for dr in range(-5, 6):
            for dc in range(-5, 6):
                rr, cc = r + dr, c + dc
                if 0 <= rr < 17 and 0 <= cc < 23:
                    a, b, w = x[0, rr, cc], y[0, rr, cc], w2[dr + 5, dc + 5]
                    m["x"] += w * a; m["y"] += w * b
                    m["xx"] += w * a * a; m["yy"] += w * b * b; m["xy"] += w * a * b
        vx, vy = m["xx"] - m["x"] ** 2, m["yy"] - m["y"] ** 2
        cov = m["xy"] - m["x"] * m["y"]
        ref = ((2 * m["x"] * m["y"] + SS.C1) * (2 * cov + SS.C2)) / \
            ((m["x"] ** 2 + m["y"] ** 2 + SS.C1) * (vx + vy + SS.C2))
        assert abs(s[r, c] - ref) <= 1e-12, (r, c)


def test_scaled_images_closed_form_with_the_published_constants():
    """x = k y: SSIM = (2k mu^2 + C1)(2k s^2 + C2) / (((k^2+1) mu^2 + C1)((k^2+1) s^2 + C2))
    with mu, s^2 the windowed mean and variance of y and Wang et al.'s constants
    C1 = (0.01 L)^2, C2 = (0.03 L)^2 for the data range L = 1 (written here, not
    read from the oracle)."""
    rng = np.random.default_rng(6)
    y = rng.uniform(0, 1, (1, 24, 24))
    k = 0.7
    mu = SS.blur(y)
    var = SS.blur(y * y) - mu * mu
    c1, c2 = (0.01 * 1.0) ** 2, (0.03 * 1.0) ** 2
    ref = (2 * k * mu * mu + c1) * (2 * k * var + c2) / (((k * k + 1) * mu * mu + c1) * ((k * k + 1) * var + c2))
    assert np.allclose(SS.ssim_map(k * y, y), ref, rtol=1e-12)
