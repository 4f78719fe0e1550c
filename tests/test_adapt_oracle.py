"""Pins of the adaptive-control oracle (Sec. 3.4 "Adaptive control of
primitives") against facts that do not come from the oracle itself:
  - coverage equals a brute-force count of the selected triangle ids;
  - view-space edge ratios equal the pinhole closed form f L / (z H) for a
    fronto-parallel triangle, and views behind the camera or off screen are
    ignored;
  - a copy plan is the identity; splitting an edge halves the parent into
    two children with the parent's area and winding whose textures carry the
    parent's (affine) texture field; the plan follows its stated rules on
    hand-made cases."""
import numpy as np
import pytest

import oracle as O
from paper_2603_27151_gb300 import inputs as I


def test_coverage_is_a_count_of_selected_ids():
    rng = np.random.default_rng(0)
    ids = [rng.integers(-1, 50, size=(2, 7, 9)).astype(np.int32), rng.integers(-1, 50, size=(3, 4)).astype(np.int32)]
    got = O.coverage(ids, 50)
    ref = np.zeros(50, np.int64)
    for a in ids:
        for x in a.reshape(-1):
            if x >= 0:
                ref[x] += 1
    assert np.array_equal(got, ref)


def _camera_on_z(W, H, f, z_eye):
    """Camera at (0, 0, z_eye) looking down -z (world), +x right."""
    cam = I.look_at([0.0, 0.0, z_eye], W, H)
    cam.fx = cam.fy = f
    return cam


def test_edge_ratio_closed_form_and_view_selection():
    # a fronto-parallel right triangle at the origin, legs 0.5 along x and y
    tri = np.array([[[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [0.0, 0.5, 0.0]]], np.float32)
    cam = _camera_on_z(640, 480, 500.0, 4.0)
    R = np.asarray(cam.R, np.float64)
    r = O.edge_ratios(tri, [cam])[0]
    # pinhole: a length L at depth z projects to f L / z pixels
    legs = [0.5 * 500.0 / 4.0 / 480, np.sqrt(0.5) * 500.0 / 4.0 / 480, 0.5 * 500.0 / 4.0 / 480]
    assert np.allclose(r, legs, rtol=1e-6)
    assert abs(abs(R[2, 2]) - 1.0) < 1e-6
    # a view from behind (the triangle behind the near plane) and an off-screen view add nothing
    behind = I.look_at([0.0, 0.0, -4.0], 640, 480)
    behind.R = cam.R.copy(); behind.t = (-np.asarray(cam.R, np.float64) @ np.array([0.0, 0.0, -4.0])).astype(np.float32)
    off = _camera_on_z(640, 480, 500.0, 4.0)
    off.cx = -2000.0
    assert np.array_equal(O.edge_ratios(tri, [cam, behind, off])[0], r)
    assert np.array_equal(O.edge_ratios(tri, [behind, off])[0], np.zeros(3, np.float32))
    # a closer view dominates the maximum
    near = _camera_on_z(640, 480, 500.0, 2.0)
    assert np.allclose(O.edge_ratios(tri, [cam, near])[0], 2.0 * r, rtol=1e-6)


def _affine_grid(verts_bary_to_val, R, C):
    n = 1 << R
    ij = np.array([(i, j) for j in range(n + 1) for i in range(n + 1 - j)]) / n
    return verts_bary_to_val(ij)


def test_copy_plan_is_identity():
    rng = np.random.default_rng(1)
    v = rng.normal(size=(5, 3, 3)).astype(np.float32)
    lv = [rng.normal(size=(5, O.level_V(R), 4)).astype(np.float32) for R in (1, 2)]
    vo, lo = O.soup_rebuild(v, lv, 1, 2, np.arange(5, dtype=np.int32) << 3)
    assert np.array_equal(vo, v) and all(np.array_equal(a, b) for a, b in zip(lo, lv))


@pytest.mark.parametrize("e", [0, 1, 2])
def test_split_children_carry_the_parent_field(e):
    v = np.array([[[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 2.0, 0.0]]], np.float32)
    coef = np.array([0.25, -0.5, 0.75], np.float64)    # value = c0 + c1 b1 + c2 b2 (dyadic: exact)

    def field(b):   # b: [..., 2] parent barycentrics (b1, b2)
        return (coef[0] + coef[1] * b[..., 0] + coef[2] * b[..., 1])[..., None].astype(np.float32)
    lv = [field(_affine_grid(lambda x: x, R, 1))[None] for R in (2, 3)]
    plan = np.array([(0 << 3) | (1 + 2 * e), (0 << 3) | (2 + 2 * e)], np.int32)
    vo, lo = O.soup_rebuild(v, lv, 2, 3, plan)
    a, b, o = e, (e + 1) % 3, (e + 2) % 3
    m = 0.5 * (v[0, a] + v[0, b])
    assert np.array_equal(vo[0], np.stack([v[0, a], m, v[0, o]]))
    assert np.array_equal(vo[1], np.stack([m, v[0, b], v[0, o]]))
    area = lambda t: 0.5 * np.cross(t[1] - t[0], t[2] - t[0])
    assert np.allclose(area(vo[0]) + area(vo[1]), area(v[0]))          # same area, same winding
    assert np.dot(area(vo[0]), area(v[0])) > 0 and np.dot(area(vo[1]), area(v[0])) > 0
    # children's grids: the parent's field at the children's grid points
    P = np.eye(3)
    Pm = 0.5 * (P[a] + P[b])
    corners = [np.stack([P[a], Pm, P[o]]), np.stack([Pm, P[b], P[o]])]
    for k in range(2):
        for R, g in zip((2, 3), lo):
            n = 1 << R
            ij = np.array([(i, j) for j in range(n + 1) for i in range(n + 1 - j)]) / n
            beta = np.stack([1 - ij[:, 0] - ij[:, 1], ij[:, 0], ij[:, 1]], -1)
            pb = beta @ corners[k]
            assert np.array_equal(g[k], field(pb[:, 1:3]))


def test_plan_rules():
    counts = np.array([5, 0, 9, 0, 3])
    ratios = np.array([[0.1, 0.3, 0.3], [0, 0, 0], [0.05, 0.0, 0.21], [0.5, 0, 0], [0.1, 0.1, 0.1]], np.float32)
    # no budget: triangles 0 (edge 1, first of the equal maxima), 2 (edge 2), 3 (edge 0) split
    p = O.adapt_plan(counts, ratios, 0.2, -1)
    assert list(p) == [0 << 3 | 3, 0 << 3 | 4, 1 << 3, 2 << 3 | 5, 2 << 3 | 6, 3 << 3 | 1, 3 << 3 | 2, 4 << 3]
    # budget 6 from 5 + 3 = 8: remove 1 (count 0, index 1: -1 -> 7), then 3 (count 0, split: -2 -> 5)
    p = O.adapt_plan(counts, ratios, 0.2, 6)
    assert list(p) == [0 << 3 | 3, 0 << 3 | 4, 2 << 3 | 5, 2 << 3 | 6, 4 << 3]
    # the threshold is strict
    assert list(O.adapt_plan(counts, ratios, 0.5, -1)) == [t << 3 for t in range(5)]


def test_library_plan_equals_the_oracle_plan():
    """ds_adapt_plan (host C++ of the library, no GPU) against the oracle's
    plan on random counts and ratios: the same integers."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_27151_gb300 import native as N
    rng = np.random.default_rng(3)
    for T, budget in [(1, -1), (50, -1), (200, 150), (200, 10), (300, 0), (64, 1000)]:
        counts = rng.integers(0, 6, size=T)
        ratios = (rng.integers(0, 8, size=(T, 3)) / 20.0).astype(np.float32)   # many ties
        got = N.adapt_plan(counts, ratios, 0.2, budget)
        assert np.array_equal(got, O.adapt_plan(counts, ratios, 0.2, budget)), (T, budget)


def test_fill_plan_rules():
    """Random-initialisation round: uncovered triangles go, then the longest
    edges of the survivors split until the target count is reached."""
    counts = np.array([4, 0, 2, 9, 1])
    ratios = np.array([[0.1, 0.4, 0.2], [0.9, 0.0, 0.0], [0.3, 0.3, 0.1], [0.05, 0.0, 0.0], [0.4, 0.1, 0.0]],
                      np.float32)
    # survivors 0, 2, 3, 4 (4); target 6: split the two longest (0: 0.4 on edge 1, 4: 0.4 on edge 0; ties by index)
    p = O.adapt_plan_fill(counts, ratios, 6)
    assert list(p) == [0 << 3 | 3, 0 << 3 | 4, 2 << 3, 3 << 3, 4 << 3 | 1, 4 << 3 | 2]
    # target below the survivors: only the removal
    assert list(O.adapt_plan_fill(counts, ratios, 2)) == [0 << 3, 2 << 3, 3 << 3, 4 << 3]
    # target far above: every survivor splits once (edge 0 of triangle 2: first of equal maxima)
    p = O.adapt_plan_fill(counts, ratios, 100)
    assert len(p) == 8 and list(p[2:4]) == [2 << 3 | 1, 2 << 3 | 2]


def test_library_fill_plan_equals_the_oracle():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_27151_gb300 import native as N
    rng = np.random.default_rng(5)
    for T, target in [(1, 5), (50, 60), (200, 150), (300, 1000), (64, 64)]:
        counts = rng.integers(0, 3, size=T)
        ratios = (rng.integers(0, 6, size=(T, 3)) / 10.0).astype(np.float32)
        got = N.adapt_plan_fill(counts, ratios, target)
        assert np.array_equal(got, O.adapt_plan_fill(counts, ratios, target)), (T, target)
