"""Pins of the deferred-shading oracle (oracle/shading.py) against facts that
do not come from the oracle itself: the orthonormality of the SH basis on
the sphere, the camera geometry of the principal ray, the special cases of
the RGBA blend, one-hot probes of every layer (operand order), the positive
homogeneity of ReLU, and central finite differences for the backward."""
import math

import numpy as np
import pytest

from oracle import shading as SH
from paper_2603_27151_gb300 import inputs as I


def _sphere_quadrature(n_theta=64, n_phi=128):
    """Gauss-Legendre in cos(theta) x uniform phi: exact for polynomials of
    low degree on the sphere."""
    u, wu = np.polynomial.legendre.leggauss(n_theta)
    phi = (np.arange(n_phi) + 0.5) * 2 * np.pi / n_phi
    ct, p = np.meshgrid(u, phi, indexing="ij")
    st = np.sqrt(1 - ct * ct)
    d = np.stack([st * np.cos(p), st * np.sin(p), ct], -1)
    w = (wu[:, None] * np.full(n_phi, 2 * np.pi / n_phi)[None, :])
    return d.reshape(-1, 3), w.reshape(-1)


def test_sh_basis_is_orthonormal_on_the_sphere():
    d, w = _sphere_quadrature()
    Y = SH.sh2(d)
    G = (Y * w[:, None]).T @ Y
    assert np.allclose(G, np.eye(9), atol=1e-10)


def test_band1_is_linear_and_band2_is_quadratic():
    """Degree-1 functions are linear in the direction and degree-2 ones
    quadratic: scaling the (unnormalised) argument scales them by s and s^2."""
    rng = np.random.default_rng(0)
    d = rng.normal(size=(50, 3))
    Y, Ys = SH.sh2(d), SH.sh2(2.0 * d)
    assert np.allclose(Ys[:, 1:4], 2.0 * Y[:, 1:4])
    assert np.allclose(Ys[:, 4:9], 4.0 * Y[:, 4:9])


def test_principal_ray_is_the_camera_forward_axis():
    cam = I.look_at([1.0, -2.0, 0.5], 64, 48)
    cam.cx, cam.cy = 20.5, 13.5               # the pixel centre (20, 13) sits on the principal point
    d = SH.view_dirs(cam)
    fwd = np.asarray(cam.R, np.float64)[2]
    assert np.allclose(d[13, 20], fwd / np.linalg.norm(fwd), atol=1e-12)
    eye = np.array([1.0, -2.0, 0.5])
    assert np.allclose(d[13, 20], -eye / np.linalg.norm(eye), atol=1e-6)   # looks at the origin
    assert np.allclose(np.linalg.norm(d, axis=-1), 1.0)


def _feat(S=2, H=5, W=7, seed=1):
    return np.random.default_rng(seed).uniform(0, 1, (S, 7, H, W))


def test_blend_special_cases():
    cam = I.look_at([0.0, 0.0, 3.0], 7, 5)
    p = SH.xavier_params(3)
    f = _feat()
    f1 = f.copy()
    f1[:, 3] = 1.0
    assert np.allclose(SH.shade(f1, cam, p), f1[:, 0:3])                # A = 1: the feature colour
    f0 = f.copy()
    f0[:, 3] = 0.0
    W1, b1, W2, b2, W3, b3 = SH.unpack(p)
    z = SH.pack(0 * W1, b1, 0 * W2, b2, 0 * W3, np.array([0.3, -1.0, 2.0]))
    sig = 1 / (1 + np.exp(-np.array([0.3, -1.0, 2.0])))
    assert np.allclose(SH.shade(f0, cam, z), sig[None, :, None, None] * np.ones((2, 3, 5, 7)))


def test_one_hot_probes_fix_every_operand_order():
    """With weights that route one input to one output through each layer,
    the output shows which input and which unit the oracle connected."""
    cam = I.look_at([0.0, 0.0, 3.0], 3, 2)
    f = np.zeros((1, 7, 2, 3))
    f[0, 5] = 0.8                                   # input 5 (a feature channel)
    W1 = np.zeros((16, 16)); W1[9, 5] = 2.0         # unit 9 <- input 5
    W2 = np.zeros((16, 16)); W2[4, 9] = 3.0         # unit 4 <- unit 9
    W3 = np.zeros((3, 16)); W3[2, 4] = 0.5          # output 2 <- unit 4
    p = SH.pack(W1, np.zeros(16), W2, np.zeros(16), W3, np.zeros(3))
    out = SH.shade(f, cam, p)                       # A = f[3] = 0: pure MLP output
    expect = 1 / (1 + np.exp(-0.5 * 3.0 * 2.0 * 0.8))
    assert np.allclose(out[0, 2], expect) and np.allclose(out[0, :2], 0.5)
    # a negative pre-activation is cut by the hidden ReLU: output sigmoid(0)
    W1n = np.zeros((16, 16)); W1n[9, 5] = -2.0
    pn = SH.pack(W1n, np.zeros(16), W2, np.zeros(16), W3, np.zeros(3))
    assert np.allclose(SH.shade(f, cam, pn), 0.5)
    # an SH input: the constant band routed to output 0
    W1 = np.zeros((16, 16)); W1[0, 7] = 1.0
    W2 = np.zeros((16, 16)); W2[0, 0] = 1.0
    W3 = np.zeros((3, 16)); W3[0, 0] = 1.0
    p = SH.pack(W1, np.zeros(16), W2, np.zeros(16), W3, np.zeros(3))
    assert np.allclose(SH.shade(f, cam, p)[0, 0], 1 / (1 + np.exp(-0.28209479177387814)))


def test_relu_rescaling_leaves_the_output_unchanged():
    cam = I.look_at([0.3, 2.0, 1.0], 6, 4)
    f = _feat(1, 4, 6, seed=5)
    W1, b1, W2, b2, W3, b3 = SH.unpack(SH.xavier_params(7))
    b1 = np.random.default_rng(2).normal(size=16)
    a = SH.shade(f, cam, SH.pack(W1, b1, W2, b2, W3, b3))
    b = SH.shade(f, cam, SH.pack(3.0 * W1, 3.0 * b1, W2 / 3.0, b2, W3, b3))
    assert np.allclose(a, b, rtol=1e-12)


def test_backward_matches_central_differences():
    cam = I.look_at([0.5, -2.0, 1.5], 5, 4)
    rng = np.random.default_rng(9)
    f = rng.uniform(0.05, 0.95, (2, 7, 4, 5))
    W1, b1, W2, b2, W3, b3 = SH.unpack(SH.xavier_params(11))
    p = SH.pack(W1, rng.normal(0, 0.3, 16), W2, rng.normal(0, 0.3, 16), W3, rng.normal(0, 0.3, 3))
    g = rng.normal(size=(2, 3, 4, 5))
    gf, gp = SH.shade_backward(f, cam, p, g)
    loss = lambda ff, pp: float(np.sum(g * SH.shade(ff, cam, pp)))
    h = 1e-6
    for idx in [(0, 0, 1, 2), (1, 3, 3, 4), (0, 6, 0, 0), (1, 4, 2, 1)]:
        e = np.zeros_like(f); e[idx] = h
        fd = (loss(f + e, p) - loss(f - e, p)) / (2 * h)
        assert abs(fd - gf[idx]) <= 1e-6 * max(1.0, abs(fd))
    for k in [0, 37, 255, 260, 300, 530, 560, 590, 594]:
        e = np.zeros_like(p); e[k] = h
        fd = (loss(f, p + e) - loss(f, p - e)) / (2 * h)
        assert abs(fd - gp[k]) <= 1e-6 * max(1.0, abs(fd)), k


def test_sh_basis_is_the_real_basis_with_the_condon_shortley_phase():
    """The oracle's basis equals the real spherical harmonics built from
    SciPy's complex ones (which carry the Condon-Shortley phase):
    Y_l0, sqrt(2) Re Y_l^m for m > 0, sqrt(2) Im Y_l^|m| for m < 0 -- this fixes
    every constant, sign and the order (m = -l..l)."""
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy.special.sph_harm_y not available")
    rng = np.random.default_rng(3)
    d = rng.normal(size=(64, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta, phi = np.arccos(d[:, 2]), np.arctan2(d[:, 1], d[:, 0])

    def real_sh(l, m):
        if m == 0:
            return sp.sph_harm_y(l, 0, theta, phi).real
        if m > 0:
            return math.sqrt(2.0) * sp.sph_harm_y(l, m, theta, phi).real
        return math.sqrt(2.0) * sp.sph_harm_y(l, -m, theta, phi).imag
    ref = np.stack([real_sh(l, m) for l in range(3) for m in range(-l, l + 1)], -1)
    assert np.allclose(SH.sh2(d), ref, atol=1e-12)
