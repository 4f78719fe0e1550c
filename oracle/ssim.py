"""CPU oracle of the photometric loss lambda L1 + (1 - lambda) L_SSIM
(Eq. 10, Sec. 3.4) per pixel, with its gradient (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use this module; the product library never loads it.  Plain
numpy in FP64.

Readings (the paper cites SSIM (Wang et al. 2004) and 3DGS for lambda =
0.8 and does not say how the loss is split per pixel for the score term of
Eq. 9, which needs a per-pixel loss value):
  - SSIM per channel with an 11 x 11 Gaussian window (sigma 1.5, weights
    normalised to sum 1), zero padding outside the image, C1 = 0.01^2,
    C2 = 0.03^2 (data range 1):
      mu_x = w * x,  sigma_x^2 = w * x^2 - mu_x^2,  sigma_xy = w * (x y) - mu_x mu_y,
      ssim = (2 mu_x mu_y + C1)(2 sigma_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2));
  - the per-pixel loss ell_p = lambda mean_c |x - y| + (1 - lambda)(1 - mean_c ssim_c(p)),
    so that the image's loss (its mean over pixels) is the paper's
    lambda L1 + (1 - lambda)(1 - SSIM); ell_p is the value the score term of
    the pixel's samples is weighted by;
  - the colour gradient is that of sum_p ell_p (non-local through the window).

Pins (tests/test_ssim_oracle.py): SSIM(x, x) = 1 and zero loss; symmetry;
the closed form for constant images away from the border; the window sums
to 1 and is separable; the map against an explicit 11 x 11 window sum at
border and interior pixels; the closed form for x = k y with Wang et al.'s
constants; the gradient against central differences.
"""
from __future__ import annotations

import numpy as np

C1 = 0.01 ** 2
C2 = 0.03 ** 2
RADIUS = 5
SIGMA = 1.5


def window1d() -> np.ndarray:
    k = np.arange(-RADIUS, RADIUS + 1, dtype=np.float64)
    g = np.exp(-k * k / (2.0 * SIGMA * SIGMA))
    return g / g.sum()


def blur(img) -> np.ndarray:
    """Zero-padded correlation of [..., H, W] with the 11 x 11 Gaussian
    (separable: the 2D window is the outer product of the 1D one)."""
    w = window1d()
    a = np.asarray(img, np.float64)
    H, W = a.shape[-2:]
    p = np.pad(a, [(0, 0)] * (a.ndim - 2) + [(RADIUS, RADIUS), (RADIUS, RADIUS)])
    h = sum(w[k] * p[..., :, k:k + W] for k in range(2 * RADIUS + 1))
    return sum(w[k] * h[..., k:k + H, :] for k in range(2 * RADIUS + 1))


def ssim_map(x, y) -> np.ndarray:
    """Per-channel SSIM map [..., C, H, W]."""
    x = np.asarray(x, np.float64); y = np.asarray(y, np.float64)
    mx, my = blur(x), blur(y)
    sxx = blur(x * x) - mx * mx
    syy = blur(y * y) - my * my
    sxy = blur(x * y) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def loss(x, y, lam: float = 0.8):
    """(ell [S, H, W], grad [S, C, H, W]): the per-pixel loss of each sample
    image x [S, C, H, W] against the target y [C, H, W], and the gradient of
    sum_p ell_p w.r.t. x."""
    x = np.asarray(x, np.float64)
    y = np.broadcast_to(np.asarray(y, np.float64), x.shape)
    C = x.shape[-3]
    mx, my = blur(x), blur(y)
    A = 2 * mx * my + C1
    B = 2 * (blur(x * y) - mx * my) + C2
    Cc = mx * mx + my * my + C1
    D = (blur(x * x) - mx * mx) + (blur(y * y) - my * my) + C2
    s = A * B / (Cc * D)
    ell = lam * np.abs(x - y).mean(-3) + (1 - lam) * (1 - s.mean(-3))
    # d s / d(raw moments m1 = w*x, m2 = w*x^2, mxy = w*(xy)), y fixed
    ds_dmu = s * (2 * my / A - 2 * mx / Cc)
    ds_dvar = -s / D
    ds_dcov = 2 * s / B
    g1 = ds_dmu + ds_dvar * (-2 * mx) + ds_dcov * (-my)
    g2 = ds_dvar
    g3 = ds_dcov
    dsum_s = blur(g1) + 2 * x * blur(g2) + y * blur(g3)      # d(sum_p s(p)) / dx(q); w is symmetric
    grad = lam * np.sign(x - y) / C - (1 - lam) * dsum_s / C
    return ell, grad
