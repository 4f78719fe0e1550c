"""Pins of the multi-resolution oracle (or_compose, or_restrict,
or_resample) against facts that do not come from the oracle itself:
  - affine reproduction: a grid sampled from an affine function of the
    position composes to the same affine function on the finest grid;
  - the hat function: one coarse vertex set to 1 composes to the closed-form
    piecewise-linear basis function of the triangulation whose diagonals run
    from (i+1, j) to (i, j+1) (this fixes the diagonal orientation, which
    affine data cannot see);
  - level 0 is the triangle's three vertices: barycentric interpolation;
  - the finest level alone is the identity; constant levels add up;
  - or_restrict is the adjoint of or_compose (dyadic data: exact in FP32);
  - resampling up then down returns the grid;
  - random levels compose to the FP64 sum of their closed-form hat-function
    expansions, to FP32 rounding, and the FP32 sum runs from the coarsest
    level up."""
import numpy as np
import pytest

import oracle as O


def _ij(R):
    """(i, j) of every vertex of the level-R grid in storage order."""
    n = 1 << R
    return np.array([(i, j) for j in range(n + 1) for i in range(n + 1 - j)])


def _affine(R, T, C, coef):
    n = 1 << R
    ij = _ij(R) / n
    g = coef[:, 0][None, None, :] + ij[None, :, 0:1] * coef[:, 1][None, None, :] + \
        ij[None, :, 1:2] * coef[:, 2][None, None, :]
    return np.broadcast_to(g, (T, len(ij), C)).astype(np.float32).copy()


def _levels_zero(r_min, r_max, T, C):
    return [np.zeros((T, O.level_V(R), C), np.float32) for R in range(r_min, r_max + 1)]


@pytest.mark.parametrize("R,r_max", [(0, 2), (1, 3), (2, 5), (3, 4)])
def test_affine_reproduction(R, r_max):
    coef = np.array([[0.25, 0.5, -0.75], [1.0, -2.0, 0.125], [-0.5, 0.375, 1.5]])   # dyadic: exact in FP32
    lv = _levels_zero(R, r_max, 2, 3)
    lv[0] = _affine(R, 2, 3, coef)
    got = O.compose(lv, R, r_max)
    assert np.array_equal(got, _affine(r_max, 2, 3, coef))


@pytest.mark.parametrize("R,r_max,u", [(2, 4, (1, 1)), (1, 3, (1, 0)), (2, 5, (2, 1)), (3, 5, (3, 2))])
def test_hat_function_fixes_the_diagonal(R, r_max, u):
    n, nf = 1 << R, 1 << r_max
    ij = _ij(R)
    k = int(np.nonzero((ij[:, 0] == u[0]) & (ij[:, 1] == u[1]))[0][0])
    lv = _levels_zero(R, r_max, 1, 1)
    lv[0][0, k, 0] = 1.0
    got = O.compose(lv, R, r_max)[0, :, 0]
    x = _ij(r_max) * (n / nf)
    dx, dy = x[:, 0] - u[0], x[:, 1] - u[1]
    hat = np.maximum(0.0, 1.0 - np.maximum(np.maximum(np.abs(dx), np.abs(dy)), np.abs(dx + dy)))
    assert np.array_equal(got, hat.astype(np.float32))
    # the other diagonal would give a different function
    other = np.maximum(0.0, 1.0 - np.maximum(np.maximum(np.abs(dx), np.abs(dy)), np.abs(dx - dy)))
    assert not np.array_equal(got, other.astype(np.float32))


def test_level0_is_the_triangle_vertices():
    vals = np.array([[0.5, -1.0], [2.0, 0.25], [-0.75, 1.5]], np.float32)   # vertex k, channel c
    lv = _levels_zero(0, 3, 1, 2)
    lv[0][0] = vals
    got = O.compose(lv, 0, 3)[0]
    b = _ij(3) / 8.0
    ref = (1 - b[:, 0] - b[:, 1])[:, None] * vals[0] + b[:, 0:1] * vals[1] + b[:, 1:2] * vals[2]
    assert np.array_equal(got, ref.astype(np.float32))


def test_finest_level_alone_is_identity_and_constants_add():
    rng = np.random.default_rng(0)
    g = rng.normal(size=(3, O.level_V(3), 4)).astype(np.float32)
    assert np.array_equal(O.compose([g], 3, 3), g)
    lv = [np.full((3, O.level_V(R), 4), 0.25 * (R + 1), np.float32) for R in range(1, 5)]
    assert np.array_equal(O.compose(lv, 1, 4), np.full((3, O.level_V(4), 4), 0.5 + 0.75 + 1.0 + 1.25, np.float32))


@pytest.mark.parametrize("r_min,r_max", [(0, 3), (2, 5), (1, 1)])
def test_restrict_is_the_adjoint_of_compose(r_min, r_max):
    rng = np.random.default_rng(r_min + 7 * r_max)
    lv = [(rng.integers(-64, 64, size=(2, O.level_V(R), 3)) / 64.0).astype(np.float32)
          for R in range(r_min, r_max + 1)]
    fine = O.compose(lv, r_min, r_max).astype(np.float64)
    g = rng.normal(size=fine.shape)
    gl = O.restrict(g, r_min, r_max)
    lhs = float(np.sum(fine * g))
    rhs = sum(float(np.sum(l.astype(np.float64) * x)) for l, x in zip(lv, gl))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_restrict_of_ones_is_the_hat_mass():
    """Each coarse vertex collects the sum of its hat function over the
    finest vertices: s^2 for an interior vertex (s = 2^(r_max - R))."""
    gl = O.restrict(np.ones((1, O.level_V(5), 1)), 2, 5)
    ij = _ij(2)
    interior = (ij[:, 0] > 0) & (ij[:, 1] > 0) & (ij.sum(1) < 4)
    assert np.allclose(gl[0][0, interior, 0], 64.0)
    for R, g in zip(range(2, 6), gl):
        assert np.isclose(g.sum(), O.level_V(5))      # partition of unity


def test_resample_up_then_down_is_identity():
    rng = np.random.default_rng(3)
    g = rng.normal(size=(2, O.level_V(2), 3)).astype(np.float32)
    up = O.resample(g, 2, 4)
    assert np.array_equal(O.resample(up, 4, 2), g)
    coef = np.array([[0.5, 0.25, -1.0]] * 3)
    assert np.array_equal(O.resample(_affine(1, 2, 3, coef), 1, 3), _affine(3, 2, 3, coef))


def _hat_expansion(g, R, r_max):
    """Level-R grid g [T][V_R][C] evaluated at the finest vertices as the sum
    of its values times their closed-form hat functions (FP64, independent
    of the oracle's cell search and interpolation)."""
    n, nf = 1 << R, 1 << r_max
    x = _ij(r_max) * (n / nf)                     # finest vertices in level-R units
    u = _ij(R)
    dx = x[:, None, 0] - u[None, :, 0]
    dy = x[:, None, 1] - u[None, :, 1]
    hat = np.maximum(0.0, 1.0 - np.maximum(np.maximum(np.abs(dx), np.abs(dy)), np.abs(dx + dy)))
    return np.einsum("fu,tuc->tfc", hat, g.astype(np.float64))


def test_compose_is_the_sum_of_the_levels_hat_expansions():
    """Random levels: every composed value equals the FP64 sum over the levels
    of their hat-function expansions at that vertex, to FP32 rounding (a
    skipped level, a wrong cell or corner, or a transposed weight fails)."""
    rng = np.random.default_rng(11)
    for r_min, r_max in [(0, 5), (2, 5), (1, 3), (0, 2)]:
        lv = [rng.normal(size=(3, O.level_V(R), 5)).astype(np.float32) for R in range(r_min, r_max + 1)]
        ref = sum(_hat_expansion(l, R, r_max) for R, l in zip(range(r_min, r_max + 1), lv))
        got = O.compose(lv, r_min, r_max)
        assert np.allclose(got, ref, rtol=0, atol=4e-7 * (r_max - r_min + 1) * 4), (r_min, r_max)


def test_compose_sums_in_level_order():
    """The levels are added in FP32 from the coarsest up: 1 + 2^-24 rounds to
    1 (ties to even), and so does the next 2^-24, whereas summing the two
    small levels first would give 1 + 2^-23."""
    lv = [np.full((1, O.level_V(R), 1), v, np.float32) for R, v in zip(range(1, 4), (1.0, 2.0 ** -24, 2.0 ** -24))]
    got = O.compose(lv, 1, 3)
    assert np.all(got == np.float32(1.0))
