"""ctypes binding of ``libdiffsoup.so`` (argument marshalling only).

The names mirror the C ABI in ``include/diffsoup.h``.  Device buffers are
passed as torch tensors (their data pointers); torch supplies the memory and
the stream, every computation runs in the library's kernels.  There is no
CPU fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libdiffsoup.so")
HEADER = os.path.join(HERE, "..", "include", "diffsoup.h")

DS_OK = 0
DS_MODE_STOCHASTIC = 0
DS_MODE_THRESHOLD_HALF = 1
DS_NO_SYNC = 0x100
DS_G_TEX, DS_G_SCORE, DS_G_INTERIOR, DS_G_EDGE = 1, 2, 4, 8
DS_G_ALL = 15
DS_REUSE_FORWARD = 0x100
DS_OVERWRITE = 0x200
DS_SHADE_N_PARAMS = 595
DS_COPY, DS_BORROW, DS_STATIC = 0, 1, 2
DS_SHADE_CUDA_CORES, DS_SHADE_TENSOR_CORES, DS_SHADE_TENSOR_CORES_WAIT_TEST = 0, 1, 2
ERRORS = {-1: "DS_ERR_INVALID_ARG", -2: "DS_ERR_OOM", -3: "DS_ERR_CUDA", -4: "DS_ERR_CAPACITY",
          -5: "DS_ERR_TIMEOUT", -6: "DS_ERR_NOT_FOUND", -7: "DS_ERR_BUSY"}


class DsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class ds_camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("near_z", ctypes.c_float)]


class ds_adam_args(ctypes.Structure):
    _fields_ = [("m", ctypes.c_void_p), ("v", ctypes.c_void_p), ("n", ctypes.c_int64), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("step", ctypes.c_int64)]


class ds_view_out(ctypes.Structure):
    _fields_ = [("gbuf", ctypes.c_void_p), ("color", ctypes.c_void_p), ("n_front", ctypes.c_void_p)]


class ds_tuning(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("depth_bits", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("chunk", ctypes.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class ds_request_stats(ctypes.Structure):
    _fields_ = [("submit_ns", ctypes.c_int64), ("launch_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64),
                ("batch", ctypes.c_int32), ("pad", ctypes.c_int32)]


class ds_view_loss(ctypes.Structure):
    _fields_ = [("target", ctypes.c_void_p), ("grad_color", ctypes.c_void_p), ("score_w", ctypes.c_void_p)]


class ds_view_gin(ctypes.Structure):
    _fields_ = [("grad_color", ctypes.c_void_p), ("score_w", ctypes.c_void_p)]


_lib = None


def load():
    """Load the library (built by ``paper_2603_27151_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libdiffsoup.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    P, i32, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32
    L.ds_version.restype = i32
    L.ds_last_error.restype = ctypes.c_char_p
    L.ds_create.argtypes = [ctypes.POINTER(P), i32]
    L.ds_create.restype = i32
    L.ds_destroy.argtypes = [P]
    L.ds_destroy.restype = None
    L.ds_soup_upload.argtypes = [P, P, P, i32, i32, i32, u32, ctypes.POINTER(i32), P]
    L.ds_soup_upload.restype = i32
    L.ds_soup_free.argtypes = [P, i32]
    L.ds_soup_free.restype = i32
    L.ds_raster_forward.argtypes = [P, i32, P, P, i32, i32, u32, P, P, P]
    L.ds_raster_forward_multi.argtypes = [P, P, P, P, i32, i32, u32, P, P, P]
    L.ds_raster_forward_multi.restype = i32
    L.ds_raster_forward.restype = i32
    L.ds_raster_backward.argtypes = [P, i32, P, i32, i32, P, P, u32, P, P, P]
    L.ds_raster_backward.restype = i32
    L.ds_raster_backward_adam.argtypes = [P, i32, P, i32, i32, P, P, u32, P, ctypes.POINTER(ds_adam_args), P]
    L.ds_raster_backward_adam.restype = i32
    L.ds_fragment_count.argtypes = [P, i32, P, i32, ctypes.POINTER(ctypes.c_int64), P]
    L.ds_fragment_count.restype = i32
    L.ds_ctx_status.argtypes = [P]
    L.ds_ctx_status.restype = i32
    L.ds_profile_enable.argtypes = [P, i32]
    L.ds_profile_enable.restype = i32
    L.ds_profile_stages.restype = i32
    L.ds_profile_read.argtypes = [P, i32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(ctypes.c_double)]
    L.ds_profile_read.restype = i32
    L.ds_profile_reset.argtypes = [P]
    L.ds_profile_reset.restype = i32
    L.ds_kernel_launches.restype = ctypes.c_int64
    L.ds_loss_l2.argtypes = [i32, i32, i32, P, P, P, P, P, ctypes.c_float, P, P]
    L.ds_loss_l2.restype = i32
    L.ds_plan_stats.argtypes = [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    L.ds_plan_stats.restype = i32
    L.ds_raster_forward_noalloc.argtypes = [P, P, i32, i32, i32, P, P, i32, i32, u32, P, P, P]
    L.ds_raster_forward_noalloc.restype = i32
    L.ds_raster_forward_devcam.argtypes = [P, i32, P, P, P, i32, i32, u32, P, P, P]
    L.ds_raster_forward_devcam.restype = i32
    L.ds_raster_backward_devcam.argtypes = [P, i32, P, P, i32, i32, P, P, u32, P, P, P]
    L.ds_raster_backward_devcam.restype = i32
    L.ds_reserve.argtypes = [P, ctypes.c_int64]
    L.ds_reserve.restype = i32
    L.ds_raster_train_l2.argtypes = [P, i32, P, P, i32, i32, u32, P, P, P, ctypes.c_float, P, u32, P, P, P]
    L.ds_raster_train_l2.restype = i32
    L.ds_raster_train_l2_devcam.argtypes = [P, i32, P, P, P, i32, i32, u32, P, P, P, ctypes.c_float, P, u32, P, P,
                                            P]
    L.ds_raster_train_l2_devcam.restype = i32
    L.ds_set_tuning.argtypes = [P, P]
    L.ds_set_tuning.restype = i32
    L.ds_get_tuning.argtypes = [P, P]
    L.ds_get_tuning.restype = i32
    L.ds_autotune.argtypes = [P, i32, P, P, i32, i32, u32, P, P, P, P, ctypes.c_float, P, P, i32, P,
                              ctypes.POINTER(ctypes.c_float), P]
    L.ds_autotune.restype = i32
    L.ds_server_create.argtypes = [i32, i32, ctypes.c_size_t, i32, ctypes.c_int64, ctypes.POINTER(P)]
    L.ds_server_create.restype = i32
    L.ds_server_add_soup.argtypes = [P, P, P, i32, i32, i32, ctypes.POINTER(i32)]
    L.ds_server_add_soup.restype = i32
    L.ds_render_request.argtypes = [P, i32, P, ctypes.c_uint64, u32, P, P, ctypes.POINTER(ctypes.c_uint64)]
    L.ds_render_request.restype = i32
    L.ds_request_wait.argtypes = [P, ctypes.c_uint64, i32, P]
    L.ds_request_wait.restype = i32
    L.ds_server_pause.argtypes = [P, i32]
    L.ds_server_pause.restype = i32
    L.ds_server_destroy.argtypes = [P]
    L.ds_server_destroy.restype = i32
    L.ds_soup_upload_levels.argtypes = [P, P, P, i32, i32, i32, i32, u32, ctypes.POINTER(i32), P]
    L.ds_soup_upload_levels.restype = i32
    L.ds_levels_compose.argtypes = [P, i32, i32, i32, i32, i32, P, P]
    L.ds_levels_compose.restype = i32
    L.ds_levels_resample.argtypes = [P, i32, i32, i32, P, i32, P]
    L.ds_levels_resample.restype = i32
    L.ds_coverage_count.argtypes = [P, P, i32, i32, i32, P, P]
    L.ds_coverage_count.restype = i32
    L.ds_edge_ratios.argtypes = [P, i32, P, i32, P, P]
    L.ds_edge_ratios.restype = i32
    L.ds_adapt_plan.argtypes = [P, P, i32, ctypes.c_float, ctypes.c_int64, P, ctypes.POINTER(i32)]
    L.ds_adapt_plan.restype = i32
    L.ds_soup_rebuild.argtypes = [P, P, P, i32, P, i32, i32, P, i32, P, P, P]
    L.ds_adapt_plan_fill.argtypes = [P, P, i32, ctypes.c_int64, P, ctypes.POINTER(i32)]
    L.ds_adapt_plan_fill.restype = i32
    L.ds_soup_rebuild.restype = i32
    L.ds_adam_step.argtypes = [P, P, P, P, ctypes.c_int64, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                               ctypes.c_float, ctypes.c_int64, P]
    L.ds_adam_step.restype = i32
    L.ds_loss_l1_ssim.argtypes = [i32, i32, i32, P, P, P, P, P, ctypes.c_float, ctypes.c_float, P, P]
    L.ds_loss_l1_ssim.restype = i32
    L.ds_shade_forward.argtypes = [P, i32, i32, P, P, P, P, P]
    L.ds_shade_forward.restype = i32
    L.ds_set_shade_path.argtypes = [P, i32]
    L.ds_set_shade_path.restype = i32
    L.ds_get_shade_path.argtypes = [P, ctypes.POINTER(i32)]
    L.ds_get_shade_path.restype = i32
    L.ds_shade_backward.argtypes = [P, i32, i32, P, P, P, P, P, P, u32, P]
    L.ds_shade_backward.restype = i32
    _lib = L
    return L


def declared_symbols(header: str = HEADER):
    """Function names declared in the public header."""
    txt = open(header).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ds_[a-z_0-9]+)\s*\(", txt)))


def _check(rc: int):
    if rc != DS_OK:
        raise DsError(rc, load().ds_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def cameras(cams):
    """Pack ``inputs.Camera`` objects into a ds_camera array."""
    arr = (ds_camera * len(cams))()
    for a, c in zip(arr, cams):
        a.width, a.height = int(c.width), int(c.height)
        a.fx, a.fy, a.cx, a.cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        R = np.asarray(c.R, np.float32).reshape(9)
        t = np.asarray(c.t, np.float32).reshape(3)
        for i in range(9):
            a.R[i] = float(R[i])
        for i in range(3):
            a.t[i] = float(t[i])
        a.near_z = float(c.near)
    return arr


class Context:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0):
        L = load()
        h = ctypes.c_void_p()
        _check(L.ds_create(ctypes.byref(h), int(device)))
        self.h = h
        self.device = device
        self._soups = {}   # soup id -> (T, C, texture floats), for the buffer checks

    def _check_views(self, soup_ids, sizes, S, gbufs=None, colors=None, n_fronts=None, grad_colors=None,
                     score_ws=None, targets=None, grad_verts=None, grad_tex=None):
        """Host-side checks of the per-view buffers (the C ABI sees raw
        pointers): sizes[v] = (W, H); gbufs int32 [S,H,W,4], n_fronts int32
        [S,H,W], score weights float32 [S,H,W], and, for a soup uploaded
        through this object, colours and colour gradients float32
        [S,C-1,H,W], targets [C-1,H,W], grad_verts 9T and grad_tex the
        texture's size; all contiguous CUDA tensors."""
        import torch
        n = len(sizes)
        if S < 1:
            return   # the library rejects the sample count itself

        def need(t, shape, dt, what):
            if t is None:
                return
            if not (t.is_cuda and t.is_contiguous() and t.dtype == dt and (shape is None or tuple(t.shape) == shape)):
                raise ValueError("%s must be a contiguous %s CUDA tensor%s" % (what, dt, "" if shape is None else
                                                                                " of shape %s" % (shape,)))
        for name, lst in (("gbufs", gbufs), ("colors", colors), ("n_fronts", n_fronts), ("grad_colors", grad_colors),
                          ("score_ws", score_ws), ("targets", targets)):
            if lst is not None and len(lst) != n:
                raise ValueError("%s: one buffer per view is required" % name)
        for v, (W, H) in enumerate(sizes):
            meta = self._soups.get(int(soup_ids[v]))
            Co = meta[1] - 1 if meta else None
            need(gbufs[v] if gbufs is not None else None, (S, H, W, 4), torch.int32, "gbufs[%d]" % v)
            need(n_fronts[v] if n_fronts is not None else None, (S, H, W), torch.int32, "n_fronts[%d]" % v)
            need(score_ws[v] if score_ws is not None else None, (S, H, W), torch.float32, "score_ws[%d]" % v)
            for name, lst, shape in (("colors", colors, (S, Co, H, W)), ("grad_colors", grad_colors, (S, Co, H, W)),
                                     ("targets", targets, (Co, H, W))):
                if lst is not None:
                    need(lst[v], shape if meta else None, torch.float32, "%s[%d]" % (name, v))
        meta = self._soups.get(int(soup_ids[0])) if n else None
        if meta is not None:
            need(grad_verts, None, torch.float32, "grad_verts")
            need(grad_tex, None, torch.float32, "grad_tex")
            if grad_verts is not None and grad_verts.numel() != 9 * meta[0]:
                raise ValueError("grad_verts must hold 9 T = %d values" % (9 * meta[0]))
            if grad_tex is not None and grad_tex.numel() != meta[2]:
                raise ValueError("grad_tex must hold the texture's %d values" % meta[2])

    def close(self):
        if self.h:
            load().ds_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- soups
    def soup_upload(self, verts, tex, grid_n: int, borrow: bool = False, static: bool = False,
                    stream=None) -> int:
        """verts: [T,3,3] float32 CUDA tensor; tex: [T,V,C] float32 CUDA tensor."""
        assert verts.is_cuda and tex.is_cuda and verts.is_contiguous() and tex.is_contiguous()
        T, V, C = tex.shape
        sid = ctypes.c_int32(-1)
        flags = (DS_BORROW if borrow else DS_COPY) | (DS_STATIC if static else 0)
        _check(load().ds_soup_upload(self.h, _ptr(verts), _ptr(tex), T, grid_n, C, flags, ctypes.byref(sid),
                                     _stream(stream)))
        self._soups[sid.value] = (int(T), int(C), int(tex.numel()))
        return sid.value

    def soup_upload_levels(self, verts, tex_levels, T: int, r_min: int, r_max: int, C: int, borrow: bool = False,
                           static: bool = False, stream=None) -> int:
        """Multi-resolution soup (ds_soup_upload_levels): tex_levels is one
        float32 CUDA tensor holding levels r_min..r_max back to back, level R
        as [T, V_R, C] (see ``level_sizes``)."""
        assert verts.is_cuda and tex_levels.is_cuda and verts.is_contiguous() and tex_levels.is_contiguous()
        assert tex_levels.numel() == sum(level_sizes(T, r_min, r_max, C))
        sid = ctypes.c_int32(-1)
        flags = (DS_BORROW if borrow else DS_COPY) | (DS_STATIC if static else 0)
        _check(load().ds_soup_upload_levels(self.h, _ptr(verts), _ptr(tex_levels), T, r_min, r_max, C, flags,
                                            ctypes.byref(sid), _stream(stream)))
        self._soups[sid.value] = (int(T), int(C), int(tex_levels.numel()))
        return sid.value

    def soup_free(self, soup_id: int):
        _check(load().ds_soup_free(self.h, soup_id))
        self._soups.pop(int(soup_id), None)

    # -------------------------------------------------------------- passes
    def raster_forward(self, soup_id, cams, seeds, S, mode, bg, gbufs, colors, n_fronts=None, stream=None):
        """gbufs[v]: int32 [S,H,W,4] (tri_id, b1, b2, depth bit patterns);
        colors[v]: float32 [S,C-1,H,W]; n_fronts[v]: int32 [S,H,W] or None."""
        n = len(cams)
        self._check_views([soup_id] * n, [(c.width, c.height) for c in cams], S, gbufs, colors, n_fronts)
        ca = cameras(cams)
        sd = (ctypes.c_uint64 * n)(*[int(x) for x in (seeds if seeds is not None else [0] * n)])
        bga = np.ascontiguousarray(bg, np.float32)
        outs = (ds_view_out * n)()
        for v in range(n):
            outs[v].gbuf = gbufs[v].data_ptr()
            outs[v].color = colors[v].data_ptr()
            outs[v].n_front = n_fronts[v].data_ptr() if n_fronts is not None and n_fronts[v] is not None else None
        _check(load().ds_raster_forward(self.h, soup_id, ca, sd, n, S, mode,
                                        bga.ctypes.data_as(ctypes.c_void_p), outs, _stream(stream)))

    def raster_forward_multi(self, soup_ids, cams, seeds, S, mode, bg, gbufs, colors, n_fronts=None, stream=None):
        """Views of different soups in one launch (ds_raster_forward_multi):
        view v renders soup soup_ids[v]; outputs as raster_forward."""
        n = len(cams)
        self._check_views(list(soup_ids), [(c.width, c.height) for c in cams], S, gbufs, colors, n_fronts)
        ids = (ctypes.c_int32 * n)(*[int(x) for x in soup_ids])
        ca = cameras(cams)
        sd = (ctypes.c_uint64 * n)(*[int(x) for x in (seeds if seeds is not None else [0] * n)])
        bga = np.ascontiguousarray(bg, np.float32)
        outs = (ds_view_out * n)()
        for v in range(n):
            outs[v].gbuf = gbufs[v].data_ptr()
            outs[v].color = colors[v].data_ptr()
            outs[v].n_front = n_fronts[v].data_ptr() if n_fronts is not None and n_fronts[v] is not None else None
        _check(load().ds_raster_forward_multi(self.h, ids, ca, sd, n, S, mode, bga.ctypes.data_as(ctypes.c_void_p),
                                              outs, _stream(stream)))

    def raster_backward(self, soup_id, cams, S, gbufs, colors, grad_colors, score_ws, flags,
                        grad_verts=None, grad_tex=None, stream=None):
        n = len(cams)
        self._check_views([soup_id] * n, [(c.width, c.height) for c in cams], S, gbufs, colors, None, grad_colors,
                          score_ws, grad_verts=grad_verts, grad_tex=grad_tex)
        ca = cameras(cams)
        fwd = (ds_view_out * n)()
        gin = (ds_view_gin * n)()
        for v in range(n):
            fwd[v].gbuf = gbufs[v].data_ptr()
            fwd[v].color = colors[v].data_ptr() if colors is not None else None
            gin[v].grad_color = grad_colors[v].data_ptr() if grad_colors is not None else None
            gin[v].score_w = score_ws[v].data_ptr() if score_ws is not None and score_ws[v] is not None else None
        _check(load().ds_raster_backward(self.h, soup_id, ca, n, S, fwd, gin, flags,
                                         _ptr(grad_verts), _ptr(grad_tex), _stream(stream)))

    def raster_backward_adam(self, soup_id, cams, S, gbufs, colors, grad_colors, score_ws, flags, m, v,
                             lr: float, step: int, grad_verts=None, beta1: float = 0.9, beta2: float = 0.999,
                             eps: float = 1e-8, stream=None):
        """ds_raster_backward_adam: the backward with one Adam step of the
        soup's own texture fused into the gradient finish (no texture gradient
        is written); m, v: float32 CUDA tensors of the texture's size."""
        import torch
        for t in (m, v):
            if t is None or t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
                raise ValueError("m and v must be contiguous float32 CUDA tensors")
        if m.numel() != v.numel():
            raise ValueError("m and v must have the same size")
        n = len(cams)
        self._check_views([soup_id] * n, [(c.width, c.height) for c in cams], S, gbufs, colors, None, grad_colors,
                          score_ws, grad_verts=grad_verts)
        ca = cameras(cams)
        fwd = (ds_view_out * n)()
        gin = (ds_view_gin * n)()
        for k in range(n):
            fwd[k].gbuf = gbufs[k].data_ptr()
            fwd[k].color = colors[k].data_ptr() if colors is not None else None
            gin[k].grad_color = grad_colors[k].data_ptr() if grad_colors is not None else None
            gin[k].score_w = score_ws[k].data_ptr() if score_ws is not None and score_ws[k] is not None else None
        args = ds_adam_args(m.data_ptr(), v.data_ptr(), m.numel(), float(lr), float(beta1), float(beta2), float(eps),
                            int(step))
        _check(load().ds_raster_backward_adam(self.h, soup_id, ca, n, S, fwd, gin, flags, _ptr(grad_verts),
                                              ctypes.byref(args), _stream(stream)))

    def set_shade_path(self, path: int):
        """Kernel of shade_forward: DS_SHADE_CUDA_CORES (FP32 FMA) or
        DS_SHADE_TENSOR_CORES (tcgen05, TF32 split into hi + lo; the default);
        DS_SHADE_TENSOR_CORES_WAIT_TEST runs the tensor-core kernel without its
        MMAs so that its bounded waits run out (DS_ERR_TIMEOUT at the next
        status check)."""
        _check(load().ds_set_shade_path(self.h, int(path)))

    def get_shade_path(self) -> int:
        p = ctypes.c_int32(-1)
        _check(load().ds_get_shade_path(self.h, ctypes.byref(p)))
        return p.value

    def shade_forward(self, cams, params, feats, rgbs, stream=None):
        """Deferred shading (ds_shade_forward): feats[v] float32 [S,7,H,W] ->
        rgbs[v] float32 [S,3,H,W] (written); params: float32 [595]."""
        n = len(cams)
        S = int(feats[0].shape[0]) if n else 1
        _check_shade(cams, S, params, [(feats, 7), (rgbs, 3)])
        arr = lambda ts: (ctypes.c_void_p * max(n, 1))(*[t.data_ptr() for t in ts])
        _check(load().ds_shade_forward(self.h, n, S, cameras(cams), _ptr(params), arr(feats), arr(rgbs),
                                       _stream(stream)))

    def shade_backward(self, cams, params, feats, grad_rgbs, grad_feats=None, grad_params=None,
                       overwrite: bool = False, stream=None):
        """Gradients of the deferred shading (ds_shade_backward); grad_feats[v]
        [S,7,H,W] and grad_params [595] are accumulated unless ``overwrite``."""
        n = len(cams)
        S = int(feats[0].shape[0]) if n else 1
        _check_shade(cams, S, params, [(feats, 7), (grad_rgbs, 3)] + ([(grad_feats, 7)] if grad_feats else []),
                     grad_params)
        arr = lambda ts: None if ts is None else (ctypes.c_void_p * max(n, 1))(*[t.data_ptr() for t in ts])
        _check(load().ds_shade_backward(self.h, n, S, cameras(cams), _ptr(params), arr(feats), arr(grad_rgbs),
                                        arr(grad_feats), _ptr(grad_params), DS_OVERWRITE if overwrite else 0,
                                        _stream(stream)))

    def soup_rebuild(self, verts, tex, T: int, grid_ns, C: int, plan, verts_out, tex_out, stream=None):
        """The soup after an adaptive-control plan (ds_soup_rebuild); plan is
        a host int32 numpy array, the tensors are float32 CUDA tensors."""
        pl = np.ascontiguousarray(plan, np.int32)
        gn = (ctypes.c_int32 * len(grid_ns))(*[int(x) for x in grid_ns])
        _check(load().ds_soup_rebuild(self.h, _ptr(verts), _ptr(tex), int(T), gn, len(grid_ns), int(C),
                                      pl.ctypes.data_as(ctypes.c_void_p), len(pl), _ptr(verts_out), _ptr(tex_out),
                                      _stream(stream)))

    def raster_forward_devcam(self, soup_id, wh, cams_dev, seeds_dev, S, mode, bg, gbufs, colors, n_fronts=None,
                              stream=None):
        """Forward with device-resident cameras (uint8 tensor of n x 76 bytes,
        the ds_camera layout) and seeds (int64 tensor [n]); wh: list of (W, H)."""
        n = len(wh)
        wha = (ctypes.c_int32 * (2 * n))(*[int(x) for p in wh for x in p])
        bga = np.ascontiguousarray(bg, np.float32)
        outs = (ds_view_out * n)()
        for v in range(n):
            outs[v].gbuf = gbufs[v].data_ptr()
            outs[v].color = colors[v].data_ptr()
            outs[v].n_front = n_fronts[v].data_ptr() if n_fronts is not None and n_fronts[v] is not None else None
        _check(load().ds_raster_forward_devcam(self.h, soup_id, wha, _ptr(cams_dev), _ptr(seeds_dev), n, S, mode,
                                               bga.ctypes.data_as(ctypes.c_void_p), outs, _stream(stream)))

    def raster_backward_devcam(self, soup_id, wh, cams_dev, S, gbufs, colors, grad_colors, score_ws, flags,
                               grad_verts=None, grad_tex=None, stream=None):
        n = len(wh)
        wha = (ctypes.c_int32 * (2 * n))(*[int(x) for p in wh for x in p])
        fwd = (ds_view_out * n)()
        gin = (ds_view_gin * n)()
        for v in range(n):
            fwd[v].gbuf = gbufs[v].data_ptr()
            fwd[v].color = colors[v].data_ptr() if colors is not None else None
            gin[v].grad_color = grad_colors[v].data_ptr() if grad_colors is not None else None
            gin[v].score_w = score_ws[v].data_ptr() if score_ws is not None and score_ws[v] is not None else None
        _check(load().ds_raster_backward_devcam(self.h, soup_id, wha, _ptr(cams_dev), n, S, fwd, gin, flags,
                                                _ptr(grad_verts), _ptr(grad_tex), _stream(stream)))

    # -------------------------------------------------------------- fused training pass
    @staticmethod
    def _outs_losses(gbufs, colors, targets, grad_colors, score_ws):
        n = len(gbufs)
        outs = (ds_view_out * n)()
        lv = (ds_view_loss * n)()
        for v in range(n):
            outs[v].gbuf = gbufs[v].data_ptr()
            outs[v].color = colors[v].data_ptr()
            outs[v].n_front = None
            lv[v].target = targets[v].data_ptr()
            lv[v].grad_color = grad_colors[v].data_ptr()
            lv[v].score_w = score_ws[v].data_ptr() if score_ws is not None and score_ws[v] is not None else None
        return outs, lv

    def train_l2(self, soup_id, cams, seeds, S, mode, bg, gbufs, colors, targets, grad_colors, score_ws, scale,
                 loss, flags, grad_verts=None, grad_tex=None, stream=None):
        """ds_raster_train_l2: forward + L2 loss + backward in one call."""
        n = len(cams)
        self._check_views([soup_id] * n, [(c.width, c.height) for c in cams], S, gbufs, colors, None, grad_colors,
                          score_ws, targets, grad_verts, grad_tex)
        ca = cameras(cams)
        sd = (ctypes.c_uint64 * n)(*[int(x) for x in (seeds if seeds is not None else [0] * n)])
        bga = np.ascontiguousarray(bg, np.float32)
        outs, lv = self._outs_losses(gbufs, colors, targets, grad_colors, score_ws)
        _check(load().ds_raster_train_l2(self.h, soup_id, ca, sd, n, S, mode, bga.ctypes.data_as(ctypes.c_void_p),
                                         outs, lv, float(scale), _ptr(loss), flags, _ptr(grad_verts), _ptr(grad_tex),
                                         _stream(stream)))

    def train_l2_devcam(self, soup_id, wh, cams_dev, seeds_dev, S, mode, bg, gbufs, colors, targets, grad_colors,
                        score_ws, scale, loss, flags, grad_verts=None, grad_tex=None, stream=None):
        n = len(wh)
        wha = (ctypes.c_int32 * (2 * n))(*[int(x) for w in wh for x in w])
        bga = np.ascontiguousarray(bg, np.float32)
        outs, lv = self._outs_losses(gbufs, colors, targets, grad_colors, score_ws)
        _check(load().ds_raster_train_l2_devcam(self.h, soup_id, wha, _ptr(cams_dev), _ptr(seeds_dev), n, S, mode,
                                                bga.ctypes.data_as(ctypes.c_void_p), outs, lv, float(scale),
                                                _ptr(loss), flags, _ptr(grad_verts), _ptr(grad_tex), _stream(stream)))

    # -------------------------------------------------------------- tuning
    def set_tuning(self, tile_w=16, depth_bits=-1, blocks_per_sm=0, chunk=256):
        t = ds_tuning(int(tile_w), int(depth_bits), int(blocks_per_sm), int(chunk))
        _check(load().ds_set_tuning(self.h, ctypes.byref(t)))

    def get_tuning(self) -> dict:
        t = ds_tuning()
        _check(load().ds_get_tuning(self.h, ctypes.byref(t)))
        return t.as_dict()

    def autotune(self, soup_id, cams, seeds, S, mode, bg, gbufs, colors, grad_colors=None, score_ws=None,
                 grad_verts=None, grad_tex=None, reps: int = 3, stream=None, targets=None, scale=1.0):
        """ds_autotune: returns (tuning dict, best ms); the tuning is set on
        this context and the outputs hold a run with it.  With `targets` the
        fused training pass is timed (grad_colors / score_ws are its outputs),
        else the forward and, with grad_colors, the backward."""
        n = len(cams)
        ca = cameras(cams)
        sd = (ctypes.c_uint64 * n)(*[int(x) for x in (seeds if seeds is not None else [0] * n)])
        bga = np.ascontiguousarray(bg, np.float32)
        outs = (ds_view_out * n)()
        for v in range(n):
            outs[v].gbuf = gbufs[v].data_ptr()
            outs[v].color = colors[v].data_ptr()
            outs[v].n_front = None
        gins = None
        lv = None
        if targets is not None:
            _, lv = self._outs_losses(gbufs, colors, targets, grad_colors, score_ws)
        elif grad_colors is not None:
            gins = (ds_view_gin * n)()
            for v in range(n):
                gins[v].grad_color = grad_colors[v].data_ptr()
                gins[v].score_w = score_ws[v].data_ptr() if score_ws is not None and score_ws[v] is not None else None
        best = ds_tuning()
        ms = ctypes.c_float(0.0)
        _check(load().ds_autotune(self.h, soup_id, ca, sd, n, S, mode, bga.ctypes.data_as(ctypes.c_void_p), outs,
                                  gins, lv, float(scale), _ptr(grad_verts), _ptr(grad_tex), int(reps),
                                  ctypes.byref(best), ctypes.byref(ms), _stream(stream)))
        return best.as_dict(), float(ms.value)

    def reserve(self, pairs: int):
        _check(load().ds_reserve(self.h, int(pairs)))

    def fragment_count(self, soup_id, cams, stream=None) -> int:
        n = len(cams)
        out = ctypes.c_int64(0)
        _check(load().ds_fragment_count(self.h, soup_id, cameras(cams), n, ctypes.byref(out), _stream(stream)))
        return out.value

    def status(self):
        _check(load().ds_ctx_status(self.h))

    def plan_stats(self):
        """(pairs, tiles) of the current binning plan."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(load().ds_plan_stats(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    # -------------------------------------------------------------- profiling
    def profile(self, on: bool = True):
        _check(load().ds_profile_enable(self.h, 1 if on else 0))

    def profile_reset(self):
        _check(load().ds_profile_reset(self.h))

    def profile_read(self) -> dict:
        """{stage: (runs, total device ms)} since the last reset."""
        L = load()
        out = {}
        for i in range(L.ds_profile_stages()):
            name = ctypes.c_char_p()
            n = ctypes.c_int64()
            ms = ctypes.c_double()
            _check(L.ds_profile_read(self.h, i, ctypes.byref(name), ctypes.byref(n), ctypes.byref(ms)))
            out[name.value.decode()] = (n.value, ms.value)
        return out


def raster_forward_noalloc(verts, tex, grid_n, cams, seeds, S, mode, bg, gbufs, colors, n_fronts=None,
                           stream=None):
    """ds_raster_forward_noalloc: the forward pass on a soup given directly,
    with no context and no allocation (library-internal fixed scratch).
    verts [T,3,3] and tex [T,V,C] float32 CUDA tensors on one device; per
    view v: gbufs[v] int32 [S,H,W,4], colors[v] float32 [S,C-1,H,W] and
    optional n_fronts[v] int32 [S,H,W], all contiguous on that device.  The
    call runs with that device current."""
    import torch
    n = len(cams)
    dev = verts.device
    for name, t, dt in (("verts", verts, torch.float32), ("tex", tex, torch.float32)):
        if not (t.is_cuda and t.device == dev and t.is_contiguous() and t.dtype == dt):
            raise ValueError("%s must be a contiguous %s tensor on %s" % (name, dt, dev))
    if tex.dim() != 3:
        raise ValueError("tex must be [T, V, C]")
    T, V, C = tex.shape
    if tuple(verts.shape) != (T, 3, 3):
        raise ValueError("verts must be [T, 3, 3] with T = tex.shape[0]")
    if V != (grid_n + 1) * (grid_n + 2) // 2:
        raise ValueError("tex.shape[1] = %d is not (grid_n+1)(grid_n+2)/2 for grid_n = %d" % (V, grid_n))
    if len(gbufs) != n or len(colors) != n or (n_fronts is not None and len(n_fronts) != n):
        raise ValueError("one output buffer per camera is required")
    for v, c in enumerate(cams):
        H, W = int(c.height), int(c.width)
        want = [(gbufs[v], (S, H, W, 4), torch.int32), (colors[v], (S, C - 1, H, W), torch.float32)]
        if n_fronts is not None and n_fronts[v] is not None:
            want.append((n_fronts[v], (S, H, W), torch.int32))
        for t, shape, dt in want:
            if not (t.is_cuda and t.device == dev and t.is_contiguous() and t.dtype == dt and tuple(t.shape) == shape):
                raise ValueError("view %d: output must be a contiguous %s tensor %s on %s" % (v, dt, shape, dev))
    sd = (ctypes.c_uint64 * n)(*[int(x) for x in (seeds if seeds is not None else [0] * n)])
    bga = np.ascontiguousarray(bg, np.float32)
    if bga.size != C - 1:
        raise ValueError("bg must hold C-1 = %d values" % (C - 1))
    outs = (ds_view_out * n)()
    for v in range(n):
        outs[v].gbuf = gbufs[v].data_ptr()
        outs[v].color = colors[v].data_ptr()
        outs[v].n_front = n_fronts[v].data_ptr() if n_fronts is not None and n_fronts[v] is not None else None
    with torch.cuda.device(dev):
        _check(load().ds_raster_forward_noalloc(_ptr(verts), _ptr(tex), T, grid_n, C, cameras(cams), sd, n, S, mode,
                                                bga.ctypes.data_as(ctypes.c_void_p), outs, _stream(stream)))


def level_V(R: int) -> int:
    """Feature vertices of the level-R grid (2^R subdivisions per edge)."""
    n = 1 << R
    return (n + 1) * (n + 2) // 2


def level_sizes(T: int, r_min: int, r_max: int, C: int):
    """Float counts of levels r_min..r_max in a multi-resolution texture."""
    return [T * level_V(R) * C for R in range(r_min, r_max + 1)]


def split_levels(tex_levels, T: int, r_min: int, r_max: int, C: int):
    """Views [T, V_R, C] of the levels of a flat multi-resolution tensor."""
    out, o = [], 0
    for R, n in zip(range(r_min, r_max + 1), level_sizes(T, r_min, r_max, C)):
        out.append(tex_levels[o:o + n].view(T, level_V(R), C))
        o += n
    return out


def levels_compose(tex_levels, T: int, r_min: int, r_max: int, C: int, out, activate: bool = False, stream=None):
    """The composed finest grid [T, V_{r_max}, C] (ds_levels_compose)."""
    _check(load().ds_levels_compose(_ptr(tex_levels), T, r_min, r_max, C, int(bool(activate)), _ptr(out),
                                    _stream(stream)))


def levels_resample(src, T: int, r_src: int, C: int, dst, r_dst: int, stream=None):
    """src [T, V_{r_src}, C] sampled at the vertices of level r_dst (ds_levels_resample)."""
    _check(load().ds_levels_resample(_ptr(src), T, r_src, C, _ptr(dst), r_dst, _stream(stream)))


def coverage_count(gbufs, T: int, counts, stream=None):
    """Pixel-samples won per triangle, added to counts (int32 CUDA [T]);
    gbufs[v]: the [S, H, W, 4] G-buffers of a forward pass."""
    n = len(gbufs)
    S = int(gbufs[0].shape[0])
    hw = (ctypes.c_int32 * (2 * n))(*[int(x) for g in gbufs for x in (g.shape[2], g.shape[1])])
    arr = (ctypes.c_void_p * n)(*[g.data_ptr() for g in gbufs])
    _check(load().ds_coverage_count(arr, hw, n, S, int(T), _ptr(counts), _stream(stream)))


def edge_ratios(verts, cams, out, stream=None):
    """[T, 3] largest view-space edge length / image height over ``cams``."""
    _check(load().ds_edge_ratios(_ptr(verts), int(verts.shape[0]), cameras(cams), len(cams), _ptr(out),
                                 _stream(stream)))


def adapt_plan(counts, ratios, threshold: float, budget: int = -1) -> np.ndarray:
    """One round's split/prune plan (ds_adapt_plan, host only) from host
    arrays counts [T] and ratios [T, 3]."""
    c = np.ascontiguousarray(counts, np.int32)
    r = np.ascontiguousarray(ratios, np.float32)
    T = len(c)
    plan = np.empty(2 * T, np.int32)
    n = ctypes.c_int32(0)
    _check(load().ds_adapt_plan(c.ctypes.data_as(ctypes.c_void_p), r.ctypes.data_as(ctypes.c_void_p), T,
                                float(threshold), int(budget), plan.ctypes.data_as(ctypes.c_void_p),
                                ctypes.byref(n)))
    return plan[:n.value].copy()


def adam_step(params, grads, m, v, lr: float, step: int, dim: int = 1, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8, stream=None):
    """One Adam (dim = 1) or VectorAdam (dim = 3) step in place (ds_adam_step);
    float32 CUDA tensors, v with numel / dim entries."""
    import torch
    for name, t in (("params", params), ("grads", grads), ("m", m), ("v", v)):
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or t.device != params.device:
            raise ValueError("%s must be a contiguous float32 CUDA tensor on the parameters' device" % name)
    n = params.numel()
    if grads.numel() != n or m.numel() != n or dim < 1 or n % dim != 0 or v.numel() != n // dim:
        raise ValueError("grads and m must match params (%d values) and v hold one value per vector of %d" % (n, dim))
    _check(load().ds_adam_step(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), params.numel(), int(dim), float(lr),
                               float(beta1), float(beta2), float(eps), int(step), _stream(stream)))


def _check_shade(cams, S, params, lists, grad_params=None):
    """Host-side shape checks of the shading calls: per view [S, k, H, W]
    float32 contiguous CUDA tensors matching the camera's size, and 595
    parameters."""
    import torch
    for t in (params, grad_params):
        if t is not None and (t.numel() != DS_SHADE_N_PARAMS or t.dtype != torch.float32 or not t.is_cuda
                              or not t.is_contiguous()):
            raise ValueError("parameters must be a contiguous float32 CUDA tensor of %d values" % DS_SHADE_N_PARAMS)
    for ts, k in lists:
        if len(ts) != len(cams):
            raise ValueError("one image per camera is required")
        for v, (t, c) in enumerate(zip(ts, cams)):
            shape = (S, k, int(c.height), int(c.width))
            if tuple(t.shape) != shape or t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
                raise ValueError("view %d: expected a contiguous float32 CUDA tensor of shape %s, got %s"
                                 % (v, shape, tuple(t.shape)))


def _check_images(colors, targets, grad_colors, score_ws):
    """Host-side shape checks of the per-view image lists of the loss calls
    (the C ABI sees raw pointers): one S and one channel count for every
    view, targets [C-1, H, W], gradients like the colours, score weights
    [S, H, W], float32 contiguous CUDA tensors."""
    import torch
    if not colors or len(targets) != len(colors):
        raise ValueError("one target per view is required")
    S, Co = int(colors[0].shape[0]), int(colors[0].shape[1])
    for v, c in enumerate(colors):
        H, W = int(c.shape[2]), int(c.shape[3])
        want = [(c, (S, Co, H, W)), (targets[v], (Co, H, W))]
        if grad_colors is not None:
            want.append((grad_colors[v], (S, Co, H, W)))
        if score_ws is not None and score_ws[v] is not None:
            want.append((score_ws[v], (S, H, W)))
        for t, shape in want:
            if tuple(t.shape) != shape or t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
                raise ValueError("view %d: expected a contiguous float32 CUDA tensor of shape %s, got %s"
                                 % (v, shape, tuple(t.shape)))


def adapt_plan_fill(counts, ratios, target: int) -> np.ndarray:
    """One round of the random-initialisation procedure (ds_adapt_plan_fill,
    host only): remove uncovered triangles, split the longest edges up to
    ``target`` triangles."""
    c = np.ascontiguousarray(counts, np.int32)
    r = np.ascontiguousarray(ratios, np.float32)
    T = len(c)
    plan = np.empty(2 * T, np.int32)
    n = ctypes.c_int32(0)
    _check(load().ds_adapt_plan_fill(c.ctypes.data_as(ctypes.c_void_p), r.ctypes.data_as(ctypes.c_void_p), T,
                                     int(target), plan.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n)))
    return plan[:n.value].copy()


def loss_l2(colors, targets, grad_colors=None, score_ws=None, loss=None, scale=1.0, stream=None):
    """Fused L2 loss (see ds_loss_l2).  colors[v] [S,C-1,H,W]; targets[v]
    [C-1,H,W]; outputs written in place; loss: 1-element float32 tensor (+=)."""
    _check_images(colors, targets, grad_colors, score_ws)
    n = len(colors)
    S, Co, H0, W0 = colors[0].shape
    hw = (ctypes.c_int32 * (2 * n))()
    arr = lambda ts: None if ts is None else (ctypes.c_void_p * n)(*[t.data_ptr() for t in ts])
    for v, c in enumerate(colors):
        hw[2 * v], hw[2 * v + 1] = int(c.shape[3]), int(c.shape[2])
    _check(load().ds_loss_l2(n, S, Co + 1, hw, arr(colors), arr(targets), arr(grad_colors), arr(score_ws),
                             float(scale), _ptr(loss), _stream(stream)))


def loss_l1_ssim(colors, targets, grad_colors=None, score_ws=None, loss=None, lam: float = 0.8, scale=1.0,
                 stream=None):
    """lambda L1 + (1 - lambda) SSIM per pixel (see ds_loss_l1_ssim); the same
    arguments as ``loss_l2``."""
    _check_images(colors, targets, grad_colors, score_ws)
    n = len(colors)
    S, Co, H0, W0 = colors[0].shape
    hw = (ctypes.c_int32 * (2 * n))()
    arr = lambda ts: None if ts is None else (ctypes.c_void_p * n)(*[t.data_ptr() for t in ts])
    for v, c in enumerate(colors):
        hw[2 * v], hw[2 * v + 1] = int(c.shape[3]), int(c.shape[2])
    _check(load().ds_loss_l1_ssim(n, S, Co + 1, hw, arr(colors), arr(targets), arr(grad_colors), arr(score_ws),
                                  float(lam), float(scale), _ptr(loss), _stream(stream)))


class Server:
    """Continuous-batching render server (``ds_server_*``)."""

    def __init__(self, device: int = 0, n_streams: int = 2, mem_budget: int = 4 << 30, max_batch: int = 16,
                 reserve_pairs: int = 1 << 22):
        L = load()
        h = ctypes.c_void_p()
        _check(L.ds_server_create(int(device), int(n_streams), int(mem_budget), int(max_batch), int(reserve_pairs),
                                  ctypes.byref(h)))
        self.h = h
        self._keep = {}   # ticket -> (out struct, bg array)

    def add_soup(self, verts, tex, grid_n: int) -> int:
        assert verts.is_cuda and tex.is_cuda and verts.is_contiguous() and tex.is_contiguous()
        T, V, C = tex.shape
        sid = ctypes.c_int32(-1)
        _check(load().ds_server_add_soup(self.h, _ptr(verts), _ptr(tex), T, grid_n, C, ctypes.byref(sid)))
        return sid.value

    def submit(self, soup_id, cam, seed, mode, bg, gbuf, color, n_front=None) -> int:
        """Queue one view (gbuf int32 [1,H,W,4], color float32 [1,C-1,H,W]);
        returns the ticket."""
        ca = cameras([cam])
        out = ds_view_out()
        out.gbuf, out.color = gbuf.data_ptr(), color.data_ptr()
        out.n_front = n_front.data_ptr() if n_front is not None else None
        bga = None if bg is None else np.ascontiguousarray(bg, np.float32)
        tk = ctypes.c_uint64(0)
        _check(load().ds_render_request(self.h, int(soup_id), ca, int(seed), int(mode),
                                        None if bga is None else bga.ctypes.data_as(ctypes.c_void_p),
                                        ctypes.byref(out), ctypes.byref(tk)))
        self._keep[tk.value] = (out, bga, gbuf, color, n_front)
        return tk.value

    def wait(self, ticket: int, timeout_ms: int = -1) -> dict:
        st = ds_request_stats()
        rc = load().ds_request_wait(self.h, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(st))
        if rc != -5:
            self._keep.pop(ticket, None)
        _check(rc)
        return {"submit_ns": st.submit_ns, "launch_ns": st.launch_ns, "done_ns": st.done_ns, "batch": st.batch}

    def pause(self, on: bool = True):
        _check(load().ds_server_pause(self.h, 1 if on else 0))

    def close(self):
        if self.h:
            _check(load().ds_server_destroy(self.h))
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_launches() -> int:
    return int(load().ds_kernel_launches())


def camera_bytes(cams) -> np.ndarray:
    """ds_camera records of ``cams`` as a uint8 array [n, 76] (for device upload)."""
    arr = cameras(cams)
    return np.frombuffer(bytes(arr), dtype=np.uint8).reshape(len(cams), ctypes.sizeof(ds_camera)).copy()


def alloc_outputs(cams, S, C, device="cuda", n_front=False):
    """Allocate per-view G-buffers [S,H,W,4] int32, colours [S,C-1,H,W] and
    optional n_front [S,H,W]."""
    import torch
    g = [torch.empty((S, c.height, c.width, 4), dtype=torch.int32, device=device) for c in cams]
    col = [torch.empty((S, C - 1, c.height, c.width), dtype=torch.float32, device=device) for c in cams]
    nf = [torch.empty((S, c.height, c.width), dtype=torch.int32, device=device) for c in cams] if n_front else None
    return g, col, nf


def split_gbuf(g):
    """(tri_id int32, bary float32 [...,2], depth float32) views of a G-buffer."""
    import torch
    tri = g[..., 0]
    f = g.view(torch.float32)
    return tri, f[..., 1:3], f[..., 3]
