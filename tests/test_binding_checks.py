"""Host-side argument checks of the Python binding (no GPU needed): the
library's C ABI sees raw pointers, so the binding refuses buffers of the
wrong shape, dtype or device before any pointer goes down."""
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_2603_27151_gb300 import native as N   # noqa: E402


def _views_checker(T=10, C=8, n_tex=None):
    """Context._check_views bound to a stand-in holding one soup (id 0)."""
    ctx = types.SimpleNamespace(_soups={0: (T, C, n_tex if n_tex is not None else T * 45 * C)})
    return lambda *a, **k: N.Context._check_views(ctx, *a, **k)


def test_view_buffers_must_be_cuda_tensors_of_the_view_shape():
    check = _views_checker()
    S, W, H = 2, 6, 4
    with pytest.raises(ValueError, match="gbufs\\[0\\]"):
        check([0], [(W, H)], S, gbufs=[torch.zeros((S, H, W, 4), dtype=torch.int32)])   # host memory
    with pytest.raises(ValueError, match="one buffer per view"):
        check([0, 0], [(W, H), (W, H)], S, gbufs=[torch.zeros(1)])


def test_sample_count_below_one_is_left_to_the_library():
    check = _views_checker()
    check([0], [(6, 4)], 0, gbufs=[torch.zeros(3)])   # no exception: the C side rejects S = 0


def test_unknown_soups_skip_the_channel_checks_only():
    check = _views_checker()
    with pytest.raises(ValueError):
        check([7], [(6, 4)], 1, gbufs=[torch.zeros((1, 4, 6, 4), dtype=torch.int32)])   # still host memory


def test_adam_step_checks_before_the_library_is_called():
    x = torch.zeros(12)
    with pytest.raises(ValueError, match="CUDA"):
        N.adam_step(x, x, x, x, 0.1, 1)   # host tensors never reach the C call
