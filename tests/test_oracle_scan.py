"""The oracle's bbox-scan (object-order) mode, used only to time the CPU
baseline, gives bit for bit the brute-force results: every forward output
and both gradients, on the 64-triangle plain workload and on bands of rows
of the 2,000-triangle batched views (8 views at mixed resolutions)."""
import numpy as np
import pytest

import oracle as O
from paper_2603_27151_gb300 import inputs as I


def _check(sc, S, rows):
    a = O.forward(sc.verts, sc.tex, sc.grid_n, sc.cams, sc.seeds, S=S, bg=sc.bg, rows=rows)
    b = O.forward(sc.verts, sc.tex, sc.grid_n, sc.cams, sc.seeds, S=S, bg=sc.bg, rows=rows, scan=True)
    for x, y in zip(a, b):
        for k in x:
            assert np.array_equal(x[k], y[k]), k
    rng = np.random.default_rng(1)
    gc = [rng.normal(size=f["color"].shape).astype(np.float32) for f in a]
    sw = [rng.uniform(0.0, 1.0, size=f["tri_id"].shape).astype(np.float32) for f in a]
    ga = O.backward(sc.verts, sc.tex, sc.grid_n, sc.cams, S, a, gc, sw, rows=rows)
    gb = O.backward(sc.verts, sc.tex, sc.grid_n, sc.cams, S, a, gc, sw, rows=rows, scan=True)
    assert np.array_equal(ga[0], gb[0]) and np.array_equal(ga[1], gb[1])
    assert np.abs(ga[0]).max() > 0 and np.abs(ga[1]).max() > 0


@pytest.mark.parametrize("S", [1, 3])
def test_scan_equals_brute_force_plain(S):
    _check(I.plain_small(), S, None)


@pytest.mark.parametrize("rows", [(0, 12), (100, 123), (235, 240)])
def test_scan_equals_brute_force_batched_rows(rows):
    _check(I.batched_views(), 2, rows)
