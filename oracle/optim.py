"""CPU oracle of the optimisers (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use this module; the product library never loads it.  Plain
numpy in FP64.

Sec. 3.4 and the supplementary "Hyperparameters": VectorAdam (Ling et al.
2022) for the vertex positions and Adam (Kingma and Ba 2015) for every other
parameter, beta1 = 0.9, beta2 = 0.999, eps = 1e-8, learning rates annealed
exponentially by a factor of 100 over the run.

Adam, per value:       m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
                       x <- x - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
VectorAdam, per vector (dim consecutive values): the same first moment per
value, but one second moment per vector from the squared norm of its
gradient, v <- b2 v + (1 - b2) |g|^2, so that the update of a vector turns
with the vector (rotation equivariance).  dim = 1 is Adam.

Pins (tests/test_optim_oracle.py): the first step and a constant gradient in
closed form, rotation equivariance of VectorAdam (and its failure for Adam),
dim = 1 equals Adam.
"""
from __future__ import annotations

import numpy as np


def adam_step(x, g, m, v, lr: float, t: int, dim: int = 1, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One step at step count t >= 1 (1-based).  x, g, m: [n]; v: [n / dim].
    Returns new (x, m, v)."""
    x = np.asarray(x, np.float64); g = np.asarray(g, np.float64)
    m = np.asarray(m, np.float64); v = np.asarray(v, np.float64)
    m = b1 * m + (1.0 - b1) * g
    g2 = (g.reshape(-1, dim) ** 2).sum(1)
    v = b2 * v + (1.0 - b2) * g2
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    x = x - lr * mhat / (np.repeat(np.sqrt(vhat), dim) + eps)
    return x, m, v


def annealed_lr(lr0: float, k: int, total: int, factor: float = 100.0) -> float:
    """Exponential annealing by ``factor`` over ``total`` steps (step k = 0..total)."""
    return lr0 * factor ** (-k / total)
