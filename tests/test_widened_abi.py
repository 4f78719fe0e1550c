"""Host-side argument checks of the widened rows' C-ABI entry points (no
GPU): every call below is rejected with DS_ERR_INVALID_ARG before any CUDA
call, and the host-only plan of the adaptive control runs on the CPU."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_27151_gb300 import native as N
    return N.load()


INVALID = -1


def test_adam_step_arguments(L):
    P = ctypes.c_void_p(16)     # never dereferenced: validation fails first
    f = ctypes.c_float
    assert L.ds_adam_step(P, P, P, P, 10, 3, f(0.1), f(0.9), f(0.999), f(1e-8), 1, None) == INVALID   # dim
    assert L.ds_adam_step(P, P, P, P, 12, 5, f(0.1), f(0.9), f(0.999), f(1e-8), 1, None) == INVALID   # dim > 4
    assert L.ds_adam_step(P, P, P, P, 12, 3, f(0.1), f(0.9), f(0.999), f(1e-8), 0, None) == INVALID   # step
    assert L.ds_adam_step(P, P, P, P, 12, 3, f(0.1), f(1.0), f(0.999), f(1e-8), 1, None) == INVALID   # beta1
    assert L.ds_adam_step(None, P, P, P, 12, 3, f(0.1), f(0.9), f(0.999), f(1e-8), 1, None) == INVALID
    assert L.ds_adam_step(P, P, P, P, -1, 1, f(0.1), f(0.9), f(0.999), f(1e-8), 1, None) == INVALID


def test_loss_and_level_arguments(L):
    P = ctypes.c_void_p(16)
    hw = (ctypes.c_int32 * 2)(64, 32)
    arr = (ctypes.c_void_p * 1)(16)
    f = ctypes.c_float
    assert L.ds_loss_l1_ssim(0, 1, 4, hw, arr, arr, None, None, f(0.8), f(1.0), None, None) == INVALID   # no views
    assert L.ds_loss_l1_ssim(1, 1, 4, hw, arr, arr, None, None, f(1.5), f(1.0), None, None) == INVALID   # lambda
    assert L.ds_loss_l1_ssim(1, 0, 4, hw, arr, arr, None, None, f(0.8), f(1.0), None, None) == INVALID   # S
    bad_hw = (ctypes.c_int32 * 2)(0, 32)
    assert L.ds_loss_l1_ssim(1, 1, 4, bad_hw, arr, arr, None, None, f(0.8), f(1.0), None, None) == INVALID
    assert L.ds_levels_compose(None, 10, 0, 3, 8, 0, P, None) == INVALID
    assert L.ds_levels_compose(P, 10, 3, 2, 8, 0, P, None) == INVALID          # r_min > r_max
    assert L.ds_levels_compose(P, 10, 0, 6, 8, 0, P, None) == INVALID          # 2^6 > 32
    assert L.ds_levels_compose(P, 0, 0, 3, 8, 0, P, None) == INVALID           # T
    assert L.ds_levels_resample(P, 10, 6, 8, P, 1, None) == INVALID
    assert L.ds_levels_resample(P, 10, 1, 17, P, 2, None) == INVALID           # C
    assert L.ds_soup_upload_levels(None, P, P, 10, 0, 3, 8, 0, ctypes.byref(ctypes.c_int32()), None) == INVALID


def test_shading_and_adaptive_arguments(L):
    P = ctypes.c_void_p(16)
    arr = (ctypes.c_void_p * 1)(16)
    hw = (ctypes.c_int32 * 2)(64, 32)
    assert L.ds_shade_forward(None, 1, 1, P, P, arr, arr, None) == INVALID      # no context
    assert L.ds_shade_backward(None, 1, 1, P, P, arr, arr, None, P, 0, None) == INVALID
    assert L.ds_coverage_count(None, hw, 1, 1, 10, P, None) == INVALID
    assert L.ds_coverage_count(arr, hw, 1, 1, 0, P, None) == INVALID           # T
    assert L.ds_edge_ratios(None, 10, P, 1, P, None) == INVALID
    plan = (ctypes.c_int32 * 1)(0)
    gn = (ctypes.c_int32 * 1)(8)
    assert L.ds_soup_rebuild(None, P, P, 1, gn, 1, 8, plan, 1, P, P, None) == INVALID


def test_adapt_plan_runs_on_the_host(L):
    from paper_2603_27151_gb300 import native as N
    counts = np.array([3, 0, 7], np.int32)
    ratios = np.array([[0.3, 0.1, 0.0], [0.0, 0.0, 0.0], [0.1, 0.25, 0.26]], np.float32)
    plan = N.adapt_plan(counts, ratios, 0.2, -1)
    assert list(plan) == [0 << 3 | 1, 0 << 3 | 2, 1 << 3, 2 << 3 | 5, 2 << 3 | 6]
    with pytest.raises(N.DsError):
        N.adapt_plan(counts, ratios, float("nan"), -1)
