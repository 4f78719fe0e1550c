"""CPU oracle of the neural deferred shading pass (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use this module; the product library never loads it.  Plain
numpy in FP64.

Sec. 3.3 "Neural deferred shading" and the supplementary "MLP Architecture":
a shared MLP maps, per pixel, the rasterised 7-channel colour feature
concatenated with the degree-2 spherical-harmonic encoding of the view
direction (7 + 9 = 16 inputs) through two 16-unit hidden layers to a colour;
the first four feature channels, read as RGBA, are blended with the MLP's
colour (a parameter-free skip connection).  Where the paper is silent this
module takes these readings:

  - view direction: the unit world-space direction of the ray from the
    camera centre through the pixel centre, R^T ((x + 0.5 - cx) / fx,
    (y + 0.5 - cy) / fy, 1) normalised;
  - SH basis: the real orthonormal degree-0..2 basis in the usual graphics
    order and signs (constants from the closed-form real harmonics);
  - activations: ReLU on both hidden layers, sigmoid on the output;
  - blend: rgb = A * feat_rgb + (1 - A) * mlp, (feat_rgb, A) = channels 0..3.

Parameters are one flat vector of 595 values: W1 [16][16] (row = output),
b1 [16], W2 [16][16], b2 [16], W3 [3][16], b3 [3].

Pins (tests/test_shading_oracle.py): SH orthonormality by quadrature on the
sphere; the SH basis equals the real harmonics built from SciPy's complex
ones (Condon-Shortley phase: every constant, sign and the order); the
principal ray is the camera's forward axis; blend special cases (A = 1 gives
the feature colour, A = 0 the MLP colour, zero weights give sigmoid(b3));
one-hot layer probes (operand order); ReLU rescaling invariance; the
backward against central differences of the forward.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT, N_FEAT, N_SH = 16, 16, 3, 7, 9
N_PARAMS = N_HID * N_IN + N_HID + N_HID * N_HID + N_HID + N_OUT * N_HID + N_OUT   # 595

_C0 = 0.28209479177387814
_C1 = 0.4886025119029199
_C2 = (1.0925484305920792, -1.0925484305920792, 0.31539156525252005, -1.0925484305920792, 0.5462742152960396)


def unpack(params):
    p = np.asarray(params, np.float64)
    assert p.size == N_PARAMS
    o = 0

    def take(n, shape):
        nonlocal o
        a = p[o:o + n].reshape(shape)
        o += n
        return a
    W1 = take(N_HID * N_IN, (N_HID, N_IN))
    b1 = take(N_HID, (N_HID,))
    W2 = take(N_HID * N_HID, (N_HID, N_HID))
    b2 = take(N_HID, (N_HID,))
    W3 = take(N_OUT * N_HID, (N_OUT, N_HID))
    b3 = take(N_OUT, (N_OUT,))
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([np.ravel(a) for a in (W1, b1, W2, b2, W3, b3)]).astype(np.float64)


def xavier_params(seed: int) -> np.ndarray:
    """Xavier-uniform weights (limit sqrt(6 / (fan_in + fan_out))), zero biases."""
    rng = np.random.default_rng(seed)
    W = [rng.uniform(-1, 1, (o, i)) * np.sqrt(6.0 / (i + o)) for (o, i) in ((16, 16), (16, 16), (3, 16))]
    return pack(W[0], np.zeros(16), W[1], np.zeros(16), W[2], np.zeros(3))


def view_dirs(cam) -> np.ndarray:
    """[H][W][3] unit world-space view directions through the pixel centres."""
    W, H = cam.width, cam.height
    x = (np.arange(W, dtype=np.float64) + 0.5 - cam.cx) / cam.fx
    y = (np.arange(H, dtype=np.float64) + 0.5 - cam.cy) / cam.fy
    dc = np.stack(np.broadcast_arrays(x[None, :], y[:, None], np.ones((H, W))), -1)   # camera frame
    R = np.asarray(cam.R, np.float64)
    dw = dc @ R          # R^T d for row vectors
    return dw / np.linalg.norm(dw, axis=-1, keepdims=True)


def sh2(d) -> np.ndarray:
    """Real SH basis up to degree 2 of unit directions d [..., 3] -> [..., 9]."""
    x, y, z = d[..., 0], d[..., 1], d[..., 2]
    return np.stack([np.full_like(x, _C0), -_C1 * y, _C1 * z, -_C1 * x,
                     _C2[0] * x * y, _C2[1] * y * z, _C2[2] * (2 * z * z - x * x - y * y), _C2[3] * x * z,
                     _C2[4] * (x * x - y * y)], -1)


def _sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def _forward(x, params):
    W1, b1, W2, b2, W3, b3 = unpack(params)
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    o = _sigmoid(h2 @ W3.T + b3)
    return z1, h1, z2, h2, o


def _inputs(feat, cam):
    """feat [S][7][H][W] -> x [S][H][W][16]."""
    f = np.moveaxis(np.asarray(feat, np.float64), 1, -1)            # [S][H][W][7]
    sh = np.broadcast_to(sh2(view_dirs(cam)), f.shape[:-1] + (N_SH,))
    return f, np.concatenate([f, sh], -1)


def shade(feat, cam, params) -> np.ndarray:
    """Shaded colour [S][3][H][W] of the feature images feat [S][7][H][W]."""
    f, x = _inputs(feat, cam)
    o = _forward(x, params)[-1]
    A = f[..., 3:4]
    rgb = A * f[..., 0:3] + (1.0 - A) * o
    return np.moveaxis(rgb, -1, 1)


def shade_backward(feat, cam, params, grad_rgb):
    """Gradients of sum(grad_rgb * shade(feat)) w.r.t. the features
    [S][7][H][W] and the parameters [595] (chain rule through the blend, the
    sigmoid, the two ReLU layers and the inputs; the SH part of the input has
    no parameter)."""
    f, x = _inputs(feat, cam)
    W1, b1, W2, b2, W3, b3 = unpack(params)
    z1, h1, z2, h2, o = _forward(x, params)
    g = np.moveaxis(np.asarray(grad_rgb, np.float64), 1, -1)        # [S][H][W][3]
    A = f[..., 3:4]
    gf = np.zeros_like(f)
    gf[..., 0:3] = A * g
    gf[..., 3] = np.sum(g * (f[..., 0:3] - o), -1)
    go = (1.0 - A) * g
    d3 = go * o * (1.0 - o)                                           # d / d(W3 h2 + b3)
    gW3 = d3.reshape(-1, N_OUT).T @ h2.reshape(-1, N_HID)
    gb3 = d3.reshape(-1, N_OUT).sum(0)
    d2 = (d3 @ W3) * (z2 > 0)
    gW2 = d2.reshape(-1, N_HID).T @ h1.reshape(-1, N_HID)
    gb2 = d2.reshape(-1, N_HID).sum(0)
    d1 = (d2 @ W2) * (z1 > 0)
    gW1 = d1.reshape(-1, N_HID).T @ x.reshape(-1, N_IN)
    gb1 = d1.reshape(-1, N_HID).sum(0)
    gx = d1 @ W1
    gf += gx[..., :N_FEAT]
    return np.moveaxis(gf, -1, 1), pack(gW1, gb1, gW2, gb2, gW3, gb3)
