"""Pins of the optimiser oracle (oracle/optim.py): closed forms of the first
step and of a constant gradient, VectorAdam's rotation equivariance (which
Adam lacks), dim = 1 reduces VectorAdam to Adam, the annealing schedule."""
import numpy as np
from scipy.spatial.transform import Rotation

from oracle import optim as OP


def test_first_step_closed_form():
    g = np.array([3.0, -4.0, 0.0, 1e-3, -2.0, 2.0])
    x0 = np.zeros(6)
    x, m, v = OP.adam_step(x0, g, np.zeros(6), np.zeros(6), 0.1, 1)
    assert np.allclose(x, -0.1 * g / (np.abs(g) + 1e-8))             # m_hat = g, v_hat = g^2
    x, m, v = OP.adam_step(x0, g, np.zeros(6), np.zeros(2), 0.1, 1, dim=3)
    n = np.linalg.norm(g.reshape(2, 3), axis=1)
    assert np.allclose(x, -0.1 * g / (np.repeat(n, 3) + 1e-8))        # the unit vector of each gradient
    assert np.allclose(np.linalg.norm(x.reshape(2, 3), axis=1), 0.1)


def test_constant_gradient_gives_constant_steps():
    g = np.array([0.5, -2.0, 1.5])
    x, m, v = np.zeros(3), np.zeros(3), np.zeros(1)
    for t in range(1, 30):
        x_new, m, v = OP.adam_step(x, g, m, v, 0.01, t, dim=3)
        assert np.allclose(x_new - x, -0.01 * g / (np.linalg.norm(g) + 1e-8), rtol=1e-12)
        x = x_new


def test_vector_adam_is_rotation_equivariant_and_adam_is_not():
    rng = np.random.default_rng(0)
    R = Rotation.from_euler("xyz", [0.3, -1.1, 2.0]).as_matrix()
    grads = rng.normal(size=(12, 5, 3))
    x0 = rng.normal(size=(5, 3))

    def run(dim, rot):
        x, m, v = x0 @ rot.T, np.zeros(15), np.zeros(15 // dim)
        x = x.reshape(-1)
        for t, g in enumerate(grads, 1):
            x, m, v = OP.adam_step(x, (g @ rot.T).reshape(-1), m, v, 0.05, t, dim=dim)
        return x.reshape(5, 3)
    assert np.allclose(run(3, R), run(3, np.eye(3)) @ R.T, atol=1e-12)
    assert not np.allclose(run(1, R), run(1, np.eye(3)) @ R.T, atol=1e-6)


def test_dim1_equals_elementwise_adam_and_annealing():
    rng = np.random.default_rng(1)
    x, g = rng.normal(size=8), rng.normal(size=8)
    a = OP.adam_step(x, g, np.full(8, 0.1), np.full(8, 0.2), 0.03, 4, dim=1)
    m = 0.9 * 0.1 + 0.1 * g
    v = 0.999 * 0.2 + 0.001 * g * g
    ref = x - 0.03 * (m / (1 - 0.9 ** 4)) / (np.sqrt(v / (1 - 0.999 ** 4)) + 1e-8)
    assert np.allclose(a[0], ref, rtol=1e-14) and np.allclose(a[1], m) and np.allclose(a[2], v)
    assert OP.annealed_lr(0.05, 0, 10000) == 0.05
    assert np.isclose(OP.annealed_lr(0.05, 10000, 10000), 0.0005)
    assert np.isclose(OP.annealed_lr(0.05, 5000, 10000), 0.005)
