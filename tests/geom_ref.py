"""Independent FP64 geometry used by the oracle pins (continuous, unsnapped).

Nothing here is shared with the oracle or the CUDA library: the pins compare
their FP32 results with these textbook formulas (pinhole projection, ray /
plane intersection, polygon clipping).
"""
import numpy as np

from paper_2603_27151_gb300.inputs import Camera


def manual_camera(width, height, f, depth):
    """Camera looking down -z at the plane z = 0 from z = depth; world x maps
    to screen right and world y to screen up; screen x = f*x/depth + W/2."""
    R = np.diag([1.0, -1.0, -1.0]).astype(np.float32)
    t = np.array([0.0, 0.0, depth], np.float32)
    return Camera(width, height, float(f), float(f), width / 2.0, height / 2.0, R, t, 0.01)


def to_cam(cam, p):
    return cam.R.astype(np.float64) @ np.asarray(p, np.float64) + cam.t.astype(np.float64)


def project(cam, pc):
    return np.array([cam.fx * pc[0] / pc[2] + cam.cx, cam.fy * pc[1] / pc[2] + cam.cy])


def ray_hit(cam, Vc, sx, sy):
    """Intersection of the ray through screen point (sx, sy) with the plane of
    the camera-space triangle Vc (3x3).  Returns (b0, b1, b2, z)."""
    d = np.array([(sx - cam.cx) / cam.fx, (sy - cam.cy) / cam.fy, 1.0])
    A = np.stack([Vc[1] - Vc[0], Vc[2] - Vc[0], -d], axis=1)
    b1, b2, lam = np.linalg.solve(A, -Vc[0])
    return 1.0 - b1 - b2, b1, b2, lam


def edge_dist(P, x):
    """Signed distances (pixels) of point x to the three edges of the 2D
    triangle P (3x2), positive inside (either orientation)."""
    area = (P[1, 0] - P[0, 0]) * (P[2, 1] - P[0, 1]) - (P[2, 0] - P[0, 0]) * (P[1, 1] - P[0, 1])
    s = 1.0 if area > 0 else -1.0
    out = []
    for i in range(3):
        a, b = P[(i + 1) % 3], P[(i + 2) % 3]
        e = (a[0] - x[0]) * (b[1] - x[1]) - (b[0] - x[0]) * (a[1] - x[1])
        out.append(s * e / np.hypot(b[0] - a[0], b[1] - a[1]))
    return np.array(out)


def clip_area(P, x0, y0, x1, y1):
    """Area of the 2D polygon P clipped to the box [x0,x1]x[y0,y1]
    (Sutherland-Hodgman, then the shoelace formula)."""
    poly = [tuple(p) for p in P]
    for axis, bound, keep_ge in ((0, x0, True), (0, x1, False), (1, y0, True), (1, y1, False)):
        if not poly:
            break
        out = []
        n = len(poly)
        for k in range(n):
            cur, nxt = poly[k], poly[(k + 1) % n]
            cin = cur[axis] >= bound if keep_ge else cur[axis] <= bound
            nin = nxt[axis] >= bound if keep_ge else nxt[axis] <= bound
            if cin:
                out.append(cur)
            if cin != nin:
                tpar = (bound - cur[axis]) / (nxt[axis] - cur[axis])
                out.append((cur[0] + tpar * (nxt[0] - cur[0]), cur[1] + tpar * (nxt[1] - cur[1])))
        poly = out
    if len(poly) < 3:
        return 0.0
    a = 0.0
    for k in range(len(poly)):
        xa, ya = poly[k]
        xb, yb = poly[(k + 1) % len(poly)]
        a += xa * yb - xb * ya
    return abs(a) * 0.5


def grid_index_table(N):
    """Texel index of every grid vertex (i, j), enumerated row by row
    (j = 0..N, then i = 0..N-j)."""
    tab = {}
    k = 0
    for j in range(N + 1):
        for i in range(N + 1 - j):
            tab[(i, j)] = k
            k += 1
    return tab
