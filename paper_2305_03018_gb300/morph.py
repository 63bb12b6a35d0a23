"""ctypes binding of the C ABI in ``include/morph.h`` (argument marshalling only).

Every function named ``morph_*`` here calls the C entry point of the same
name.  The small :class:`Context` helper turns torch tensors into the C
structs (device pointers, strides, the current CUDA stream) and allocates
the outputs with torch; every step of the computation runs in the library's
CUDA kernels.  There is no CPU fallback: if the library is missing, loading
fails with an error.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libmorph_gb300.so")

MORPH_OK, MORPH_E_INVAL, MORPH_E_RANGE, MORPH_E_NOMEM, MORPH_E_PRECISION, MORPH_E_CUDA, MORPH_E_TIMEOUT, \
    MORPH_E_UNSUPPORTED = range(8)
MORPH_U8, MORPH_U16, MORPH_I32 = 0, 1, 2
MORPH_AUTO, MORPH_DIRECT_FP8, MORPH_FFT_F32, MORPH_FFT_F64, MORPH_NTT = 0, 1, 2, 3, 4
MORPH_F_ALLOW_UNPROVEN_F32, MORPH_F_VALIDATE, MORPH_F_AUTOTUNE = 1, 2, 4
METHODS = {"auto": MORPH_AUTO, "direct_fp8": MORPH_DIRECT_FP8, "fft_f32": MORPH_FFT_F32, "fft_f64": MORPH_FFT_F64,
           "ntt": MORPH_NTT}


class morph_image(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int), ("n", ctypes.c_int), ("h", ctypes.c_int),
                ("w", ctypes.c_int), ("row_stride", ctypes.c_int64), ("batch_stride", ctypes.c_int64),
                ("L", ctypes.c_int)]


class morph_se(ctypes.Structure):
    _fields_ = [("kh", ctypes.c_int), ("kw", ctypes.c_int), ("oy", ctypes.c_int), ("ox", ctypes.c_int),
                ("mask", ctypes.POINTER(ctypes.c_uint8)), ("offset", ctypes.POINTER(ctypes.c_int32))]


class morph_se_dev(ctypes.Structure):
    _fields_ = [("kh", ctypes.c_int), ("kw", ctypes.c_int), ("oy", ctypes.c_int), ("ox", ctypes.c_int),
                ("mask", ctypes.POINTER(ctypes.c_uint8)), ("offset", ctypes.c_void_p), ("max_offset", ctypes.c_int)]


class morph_volume(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int), ("n", ctypes.c_int), ("d", ctypes.c_int),
                ("h", ctypes.c_int), ("w", ctypes.c_int), ("row_stride", ctypes.c_int64),
                ("slice_stride", ctypes.c_int64), ("volume_stride", ctypes.c_int64), ("L", ctypes.c_int)]


class morph_se3d(ctypes.Structure):
    _fields_ = [("kd", ctypes.c_int), ("kh", ctypes.c_int), ("kw", ctypes.c_int), ("oz", ctypes.c_int),
                ("oy", ctypes.c_int), ("ox", ctypes.c_int), ("mask", ctypes.POINTER(ctypes.c_uint8)),
                ("offset", ctypes.POINTER(ctypes.c_int32))]


class morph_opts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("flags", ctypes.c_int), ("count_err", ctypes.c_void_p)]


class morph_plan_info(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("R", ctypes.c_int), ("taps", ctypes.c_int),
                ("f32_bound", ctypes.c_double), ("f64_bound", ctypes.c_double),
                ("fft_nx", ctypes.c_int), ("fft_ny", ctypes.c_int), ("groups", ctypes.c_int),
                ("passes", ctypes.c_int), ("tile_w", ctypes.c_int), ("tile_h", ctypes.c_int),
                ("est_flop", ctypes.c_double), ("workspace_bytes", ctypes.c_size_t),
                ("unit_tiles", ctypes.c_int), ("unit_blocks", ctypes.c_int),
                ("k_steps", ctypes.c_int), ("level_chunks", ctypes.c_int), ("ring_stages", ctypes.c_int),
                ("unit_queue", ctypes.c_int)]


class morph_problem(ctypes.Structure):
    _fields_ = [("f", morph_image), ("se", morph_se), ("op", ctypes.c_int), ("out", ctypes.c_void_p),
                ("out_count", ctypes.c_void_p)]


class morph_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double)]


# Every entry point include/morph.h declares, with its C signature.
_P = ctypes.c_void_p
_SIGS = {
    "morph_ctx_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "morph_ctx_destroy": (ctypes.c_int, [_P]),
    "morph_plan_query": (ctypes.c_int, [_P, ctypes.POINTER(morph_image), ctypes.POINTER(morph_se), ctypes.c_int,
                                        ctypes.POINTER(morph_opts), ctypes.POINTER(morph_plan_info)]),
    "morph_dilate": (ctypes.c_int, [_P, ctypes.POINTER(morph_image), ctypes.POINTER(morph_se), _P, _P,
                                    ctypes.POINTER(morph_opts), _P]),
    "morph_erode": (ctypes.c_int, [_P, ctypes.POINTER(morph_image), ctypes.POINTER(morph_se), _P, _P,
                                   ctypes.POINTER(morph_opts), _P]),
    "morph_dilate3d": (ctypes.c_int, [_P, ctypes.POINTER(morph_volume), ctypes.POINTER(morph_se3d), _P, _P,
                                      ctypes.POINTER(morph_opts), _P]),
    "morph_erode3d": (ctypes.c_int, [_P, ctypes.POINTER(morph_volume), ctypes.POINTER(morph_se3d), _P, _P,
                                     ctypes.POINTER(morph_opts), _P]),
    "morph_open": (ctypes.c_int, [_P, ctypes.POINTER(morph_image), ctypes.POINTER(morph_se), _P,
                                  ctypes.POINTER(morph_opts), _P]),
    "morph_close": (ctypes.c_int, [_P, ctypes.POINTER(morph_image), ctypes.POINTER(morph_se), _P,
                                   ctypes.POINTER(morph_opts), _P]),
    "morph_gradient": (ctypes.c_int, [_P, ctypes.POINTER(morph_image), ctypes.POINTER(morph_se), _P,
                                      ctypes.POINTER(morph_opts), _P]),
    "morph_dilate_backward": (ctypes.c_int, [_P, ctypes.POINTER(morph_image), ctypes.POINTER(morph_se), _P, _P, _P,
                                             _P, _P, _P]),
    "morph_erode_backward": (ctypes.c_int, [_P, ctypes.POINTER(morph_image), ctypes.POINTER(morph_se), _P, _P, _P,
                                            _P, _P, _P]),
    "morph_dilate_dev_se": (ctypes.c_int, [_P, ctypes.POINTER(morph_image), ctypes.POINTER(morph_se_dev), _P, _P, _P]),
    "morph_erode_dev_se": (ctypes.c_int, [_P, ctypes.POINTER(morph_image), ctypes.POINTER(morph_se_dev), _P, _P, _P]),
    "morph_dilate_backward_dev_se": (ctypes.c_int, [_P, ctypes.POINTER(morph_image), ctypes.POINTER(morph_se_dev),
                                                    _P, _P, _P, _P, _P, _P]),
    "morph_erode_backward_dev_se": (ctypes.c_int, [_P, ctypes.POINTER(morph_image), ctypes.POINTER(morph_se_dev),
                                                   _P, _P, _P, _P, _P, _P]),
    "morph_run_batch": (ctypes.c_int, [_P, ctypes.POINTER(morph_problem), ctypes.c_int, ctypes.POINTER(morph_opts),
                                       _P]),
    "morph_batch_capture": (ctypes.c_int, [_P, ctypes.POINTER(morph_problem), ctypes.c_int,
                                           ctypes.POINTER(morph_opts), ctypes.POINTER(ctypes.c_void_p)]),
    "morph_batch_launch": (ctypes.c_int, [_P, _P]),
    "morph_batch_destroy": (ctypes.c_int, [_P]),
    "morph_workspace_size": (ctypes.c_int, [_P, ctypes.POINTER(morph_image), ctypes.POINTER(morph_se), ctypes.c_int,
                                            ctypes.POINTER(morph_opts), ctypes.POINTER(ctypes.c_size_t)]),
    "morph_ctx_set_cache_limit": (ctypes.c_int, [_P, ctypes.c_size_t]),
    "morph_ctx_cache_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int)]),
    "morph_stream_check": (ctypes.c_int, [_P, _P]),
    "morph_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "morph_launch_count": (ctypes.c_uint64, [_P]),
    "morph_mma_count": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    "morph_ctx_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "morph_band_work": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    "morph_tc_fp8_peak": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "morph_run_noalloc": (ctypes.c_int, [ctypes.POINTER(morph_image), ctypes.POINTER(morph_se), ctypes.c_int, _P, _P,
                                         _P, _P]),
    "morph_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "morph_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(morph_kernel_time), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int)]),
}

_lock = threading.Lock()
_lib = None


def load_library(path: Optional[str] = None):
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built: {p} is missing (run __graft_entry__.build())")
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class MorphError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load_library().morph_strerror(status)
        super().__init__(f"{where}: status {status} ({msg.decode() if msg else '?'})")
        self.status = status


def check(status: int, where: str):
    if status != MORPH_OK:
        raise MorphError(status, where)


# ------------------------------------------------- C entry points, same names
def morph_ctx_create(device: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    check(load_library().morph_ctx_create(int(device), ctypes.byref(h)), "morph_ctx_create")
    return h


def morph_ctx_destroy(ctx) -> int:
    return load_library().morph_ctx_destroy(ctx)


def morph_plan_query(ctx, image, se, op, opts=None):
    info = morph_plan_info()
    check(load_library().morph_plan_query(ctx, ctypes.byref(image), ctypes.byref(se), int(op),
                                          ctypes.byref(opts) if opts is not None else None, ctypes.byref(info)),
          "morph_plan_query")
    return info


def morph_dilate(ctx, image, se, out_ptr, cnt_ptr, opts, stream) -> int:
    return load_library().morph_dilate(ctx, ctypes.byref(image), ctypes.byref(se), out_ptr, cnt_ptr,
                                       ctypes.byref(opts) if opts is not None else None, stream)


def morph_erode(ctx, image, se, out_ptr, cnt_ptr, opts, stream) -> int:
    return load_library().morph_erode(ctx, ctypes.byref(image), ctypes.byref(se), out_ptr, cnt_ptr,
                                      ctypes.byref(opts) if opts is not None else None, stream)


def morph_dilate3d(ctx, volume, se, out_ptr, cnt_ptr, opts, stream) -> int:
    return load_library().morph_dilate3d(ctx, ctypes.byref(volume), ctypes.byref(se), out_ptr, cnt_ptr,
                                         ctypes.byref(opts) if opts is not None else None, stream)


def morph_erode3d(ctx, volume, se, out_ptr, cnt_ptr, opts, stream) -> int:
    return load_library().morph_erode3d(ctx, ctypes.byref(volume), ctypes.byref(se), out_ptr, cnt_ptr,
                                        ctypes.byref(opts) if opts is not None else None, stream)


def morph_open(ctx, image, se, out_ptr, opts, stream) -> int:
    return load_library().morph_open(ctx, ctypes.byref(image), ctypes.byref(se), out_ptr,
                                     ctypes.byref(opts) if opts is not None else None, stream)


def morph_close(ctx, image, se, out_ptr, opts, stream) -> int:
    return load_library().morph_close(ctx, ctypes.byref(image), ctypes.byref(se), out_ptr,
                                      ctypes.byref(opts) if opts is not None else None, stream)


def morph_gradient(ctx, image, se, out_ptr, opts, stream) -> int:
    return load_library().morph_gradient(ctx, ctypes.byref(image), ctypes.byref(se), out_ptr,
                                         ctypes.byref(opts) if opts is not None else None, stream)


def morph_dilate_backward(ctx, image, se, d_ptr, cd_ptr, g_ptr, gin_ptr, gse_ptr, stream) -> int:
    return load_library().morph_dilate_backward(ctx, ctypes.byref(image), ctypes.byref(se), d_ptr, cd_ptr, g_ptr,
                                                gin_ptr, gse_ptr, stream)


def morph_erode_backward(ctx, image, se, e_ptr, ce_ptr, g_ptr, gin_ptr, gse_ptr, stream) -> int:
    return load_library().morph_erode_backward(ctx, ctypes.byref(image), ctypes.byref(se), e_ptr, ce_ptr, g_ptr,
                                               gin_ptr, gse_ptr, stream)


def morph_ctx_set_cache_limit(ctx, nbytes) -> int:
    return load_library().morph_ctx_set_cache_limit(ctx, int(nbytes))


def morph_ctx_cache_info(ctx):
    """(device bytes held by the plan cache, number of cached plans)."""
    b, n = ctypes.c_size_t(0), ctypes.c_int(0)
    check(load_library().morph_ctx_cache_info(ctx, ctypes.byref(b), ctypes.byref(n)), "morph_ctx_cache_info")
    return int(b.value), int(n.value)


def morph_workspace_size(ctx, image, se, op, opts) -> int:
    """Device workspace (bytes) a call would use; op 0/1 dilate/erode, 2/3 their backward."""
    out = ctypes.c_size_t(0)
    check(load_library().morph_workspace_size(ctx, ctypes.byref(image), ctypes.byref(se), int(op),
                                              ctypes.byref(opts) if opts is not None else None, ctypes.byref(out)),
          "morph_workspace_size")
    return int(out.value)


def morph_run_batch(ctx, problems, opts, stream) -> int:
    arr = (morph_problem * len(problems))(*problems)
    return load_library().morph_run_batch(ctx, arr, len(problems), ctypes.byref(opts) if opts is not None else None,
                                          stream)


def morph_batch_capture(ctx, problems, opts):
    arr = (morph_problem * len(problems))(*problems)
    h = ctypes.c_void_p()
    check(load_library().morph_batch_capture(ctx, arr, len(problems),
                                             ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)),
          "morph_batch_capture")
    return h


def morph_batch_launch(batch, stream) -> int:
    return load_library().morph_batch_launch(batch, stream)


def morph_batch_destroy(batch) -> int:
    return load_library().morph_batch_destroy(batch)


def morph_stream_check(ctx, stream) -> int:
    return load_library().morph_stream_check(ctx, stream)


def morph_strerror(status: int) -> str:
    r = load_library().morph_strerror(int(status))
    return r.decode() if r else ""


def morph_launch_count(ctx) -> int:
    return int(load_library().morph_launch_count(ctx))


def morph_dilate_dev_se(ctx, image, se, out_ptr, cnt_ptr, stream) -> int:
    return load_library().morph_dilate_dev_se(ctx, ctypes.byref(image), ctypes.byref(se), out_ptr, cnt_ptr, stream)


def morph_erode_dev_se(ctx, image, se, out_ptr, cnt_ptr, stream) -> int:
    return load_library().morph_erode_dev_se(ctx, ctypes.byref(image), ctypes.byref(se), out_ptr, cnt_ptr, stream)


def morph_dilate_backward_dev_se(ctx, image, se, d_ptr, cd_ptr, g_ptr, gin_ptr, gse_ptr, stream) -> int:
    return load_library().morph_dilate_backward_dev_se(ctx, ctypes.byref(image), ctypes.byref(se), d_ptr, cd_ptr,
                                                       g_ptr, gin_ptr, gse_ptr, stream)


def morph_erode_backward_dev_se(ctx, image, se, e_ptr, ce_ptr, g_ptr, gin_ptr, gse_ptr, stream) -> int:
    return load_library().morph_erode_backward_dev_se(ctx, ctypes.byref(image), ctypes.byref(se), e_ptr, ce_ptr,
                                                      g_ptr, gin_ptr, gse_ptr, stream)


def morph_ctx_set_wait_limit(ctx, ns: int) -> int:
    return load_library().morph_ctx_set_wait_limit(ctx, int(ns))


def morph_band_work(ctx) -> int:
    v = ctypes.c_uint64(0)
    check(load_library().morph_band_work(ctx, ctypes.byref(v)), "morph_band_work")
    return int(v.value)


def morph_mma_count(ctx) -> int:
    v = ctypes.c_uint64(0)
    check(load_library().morph_mma_count(ctx, ctypes.byref(v)), "morph_mma_count")
    return int(v.value)


def morph_tc_fp8_peak(ctx) -> float:
    v = ctypes.c_double(0.0)
    check(load_library().morph_tc_fp8_peak(ctx, ctypes.byref(v)), "morph_tc_fp8_peak")
    return float(v.value)


def morph_run_noalloc(image, se, op, out_ptr, cnt_ptr, status_ptr, stream) -> int:
    """Allocation-free dilation (op 0) / erosion (op 1); see include/morph.h."""
    return load_library().morph_run_noalloc(ctypes.byref(image), ctypes.byref(se), int(op), out_ptr, cnt_ptr,
                                            status_ptr, stream)


def morph_profile_enable(ctx, on: bool) -> int:
    return load_library().morph_profile_enable(ctx, 1 if on else 0)


def morph_profile_read(ctx):
    """Per-kernel totals {name: (launches, total_ms)} of the recorded launches."""
    cap = 64
    arr = (morph_kernel_time * cap)()
    n = ctypes.c_int(0)
    check(load_library().morph_profile_read(ctx, arr, cap, ctypes.byref(n)), "morph_profile_read")
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(min(n.value, cap))}


# ------------------------------------------------------------ torch helpers
_DT = {"uint8": MORPH_U8, "uint16": MORPH_U16, "int32": MORPH_I32}


def make_image(t, L: int) -> morph_image:
    """C view of a CUDA integer tensor of shape [N, H, W] (or [H, W])."""
    import torch
    if t.dim() == 2:
        t = t.unsqueeze(0)
    if t.dim() != 3 or not t.is_cuda:
        raise ValueError("image must be a CUDA tensor [N, H, W] or [H, W]")
    name = str(t.dtype).replace("torch.", "")
    if name not in _DT:
        raise ValueError(f"unsupported image dtype {t.dtype}")
    if t.stride(2) != 1:
        raise ValueError("image columns must be contiguous")
    img = morph_image()
    img.data = t.data_ptr()
    img.dtype = _DT[name]
    img.n, img.h, img.w = (int(s) for s in t.shape)
    # a size-1 dimension may carry any stride (0 after a broadcasting view): use the packed one
    img.row_stride = int(t.stride(1)) if img.h > 1 else img.w
    img.batch_stride = int(t.stride(0)) if img.n > 1 else img.h * img.row_stride
    img.L = int(L)
    return img


def make_volume(t, L: int) -> morph_volume:
    """C view of a CUDA integer tensor of shape [N, D, H, W] (or [D, H, W])."""
    if t.dim() == 3:
        t = t.unsqueeze(0)
    if t.dim() != 4 or not t.is_cuda:
        raise ValueError("volume must be a CUDA tensor [N, D, H, W] or [D, H, W]")
    name = str(t.dtype).replace("torch.", "")
    if name not in _DT:
        raise ValueError(f"unsupported volume dtype {t.dtype}")
    if t.stride(3) != 1:
        raise ValueError("volume columns must be contiguous")
    v = morph_volume()
    v.data = t.data_ptr()
    v.dtype = _DT[name]
    v.n, v.d, v.h, v.w = (int(s) for s in t.shape)
    v.row_stride = int(t.stride(2)) if v.h > 1 else v.w
    v.slice_stride = int(t.stride(1)) if v.d > 1 else v.h * v.row_stride
    v.volume_stride = int(t.stride(0)) if v.n > 1 else v.d * v.slice_stride
    v.L = int(L)
    return v


class SE3DView:
    """Host arrays of a 3-D SE kept alive next to the C struct."""

    def __init__(self, mask, offset, origin):
        self.mask = np.ascontiguousarray(np.asarray(mask) != 0, dtype=np.uint8)
        self.offset = np.ascontiguousarray(np.asarray(offset), dtype=np.int32)
        if self.mask.ndim != 3 or self.offset.shape != self.mask.shape:
            raise ValueError("mask and offset must be 3-D arrays of one shape")
        self.c = morph_se3d()
        self.c.kd, self.c.kh, self.c.kw = (int(s) for s in self.mask.shape)
        self.c.oz, self.c.oy, self.c.ox = (int(o) for o in origin)
        self.c.mask = self.mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        self.c.offset = self.offset.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


class SEView:
    """Host arrays of an SE kept alive next to the C struct that points at them."""

    def __init__(self, mask, offset, origin):
        self.mask = np.ascontiguousarray(np.asarray(mask) != 0, dtype=np.uint8)
        self.offset = np.ascontiguousarray(np.asarray(offset), dtype=np.int32)
        if self.mask.ndim != 2 or self.offset.shape != self.mask.shape:
            raise ValueError("mask and offset must be 2-D arrays of one shape")
        self.c = morph_se()
        self.c.kh, self.c.kw = (int(s) for s in self.mask.shape)
        self.c.oy, self.c.ox = int(origin[0]), int(origin[1])
        self.c.mask = self.mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        self.c.offset = self.offset.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


class SEDevView:
    """An SE whose offsets are a CUDA int32 tensor [kh, kw] (a learnable layer's
    parameter); the host mask is kept alive next to the C struct."""

    def __init__(self, mask, offset_t, origin, max_offset: int):
        self.mask = np.ascontiguousarray(np.asarray(mask) != 0, dtype=np.uint8)
        if offset_t.dtype != __import__("torch").int32 or not offset_t.is_cuda or not offset_t.is_contiguous():
            raise ValueError("device offsets must be a contiguous CUDA int32 tensor")
        if tuple(offset_t.shape) != self.mask.shape:
            raise ValueError("mask and offsets must have one shape [kh, kw]")
        self.offset_t = offset_t
        self.c = morph_se_dev()
        self.c.kh, self.c.kw = (int(s) for s in self.mask.shape)
        self.c.oy, self.c.ox = int(origin[0]), int(origin[1])
        self.c.mask = self.mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        self.c.offset = offset_t.data_ptr()
        self.c.max_offset = int(max_offset)


def se_view(se) -> SEView:
    """Accepts a workloads.SE-like object (mask, offset, origin) or a tuple."""
    if isinstance(se, SEView):
        return se
    if isinstance(se, tuple):
        return SEView(*se)
    return SEView(se.mask, se.offset, se.origin)


def make_opts(method="auto", allow_unproven_f32=False, validate=False, count_err=None, autotune=False) -> morph_opts:
    o = morph_opts()
    o.method = METHODS[method] if isinstance(method, str) else int(method)
    o.flags = ((MORPH_F_ALLOW_UNPROVEN_F32 if allow_unproven_f32 else 0) | (MORPH_F_VALIDATE if validate else 0) |
               (MORPH_F_AUTOTUNE if autotune else 0))
    o.count_err = count_err.data_ptr() if count_err is not None else None
    return o


def current_stream_handle(device=None):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class Context:
    """One library context per CUDA device (not thread-safe)."""

    def __init__(self, device: int = 0):
        import torch
        torch.cuda.init()
        self.device = int(device)
        with torch.cuda.device(self.device):
            self.handle = morph_ctx_create(self.device)

    def close(self):
        if getattr(self, "handle", None):
            morph_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- forward -------------------------------------------------------------
    def _run(self, op, f, L, se, method, count, stream, allow_unproven_f32=False, count_err=None, out=None,
             out_count=None, autotune=False):
        import torch
        img = make_image(f, L)
        sv = se_view(se)
        shape = (img.n, img.h, img.w)
        if out is None:
            out = torch.empty(shape, dtype=torch.int32, device=f.device)
        if count and out_count is None:
            out_count = torch.empty(shape, dtype=torch.int32, device=f.device)
        opts = make_opts(method, allow_unproven_f32, count_err is not None, count_err, autotune)
        st = stream if stream is not None else current_stream_handle(f.device)
        fn = morph_dilate if op == 0 else morph_erode
        check(fn(self.handle, img, sv.c, out.data_ptr(), out_count.data_ptr() if count else None, opts, st),
              "morph_dilate" if op == 0 else "morph_erode")
        return (out, out_count) if count else out

    def dilate(self, f, L, se, method="auto", count=False, stream=None, **kw):
        return self._run(0, f, L, se, method, count, stream, **kw)

    def erode(self, f, L, se, method="auto", count=False, stream=None, **kw):
        return self._run(1, f, L, se, method, count, stream, **kw)

    def morph_dev_se(self, op, f, L, sev, count=False, stream=None, out=None, out_count=None):
        """Dilation (op 0) or erosion (op 1) by an SEDevView (FP8 route, no host copy of the offsets)."""
        import torch
        img = make_image(f, L)
        shape = (img.n, img.h, img.w)
        if out is None:
            out = torch.empty(shape, dtype=torch.int32, device=f.device)
        if count and out_count is None:
            out_count = torch.empty(shape, dtype=torch.int32, device=f.device)
        st = stream if stream is not None else current_stream_handle(f.device)
        fn = morph_dilate_dev_se if op == 0 else morph_erode_dev_se
        check(fn(self.handle, img, sev.c, out.data_ptr(), out_count.data_ptr() if count else None, st),
              "morph_dilate_dev_se" if op == 0 else "morph_erode_dev_se")
        return (out, out_count) if count else out

    def _run3d(self, op, f, L, mask, offset, origin, method, count, stream):
        import torch
        vol = make_volume(f, L)
        sv = SE3DView(mask, offset, origin)
        shape = (vol.n, vol.d, vol.h, vol.w)
        out = torch.empty(shape, dtype=torch.int32, device=f.device)
        cnt = torch.empty(shape, dtype=torch.int32, device=f.device) if count else None
        st = stream if stream is not None else current_stream_handle(f.device)
        fn = morph_dilate3d if op == 0 else morph_erode3d
        check(fn(self.handle, vol, sv.c, out.data_ptr(), cnt.data_ptr() if count else None, make_opts(method), st),
              "morph_dilate3d" if op == 0 else "morph_erode3d")
        return (out, cnt) if count else out

    def dilate3d(self, f, L, mask, offset, origin, method="auto", count=False, stream=None):
        """3-D dilation of a [N, D, H, W] (or [D, H, W]) volume by a [kd, kh, kw] SE."""
        return self._run3d(0, f, L, mask, offset, origin, method, count, stream)

    def erode3d(self, f, L, mask, offset, origin, method="auto", count=False, stream=None):
        """3-D erosion of a [N, D, H, W] (or [D, H, W]) volume by a [kd, kh, kw] SE."""
        return self._run3d(1, f, L, mask, offset, origin, method, count, stream)

    def composite(self, which, f, L, se, method="auto", stream=None, out=None):
        """which: 'open' | 'close' | 'gradient'."""
        import torch
        img = make_image(f, L)
        sv = se_view(se)
        if out is None:
            out = torch.empty((img.n, img.h, img.w), dtype=torch.int32, device=f.device)
        fn = {"open": morph_open, "close": morph_close, "gradient": morph_gradient}[which]
        st = stream if stream is not None else current_stream_handle(f.device)
        check(fn(self.handle, img, sv.c, out.data_ptr(), make_opts(method), st), "morph_" + which)
        return out

    def workspace_size(self, f, L, se, op=0, method="auto", allow_unproven_f32=False):
        """Bytes of device workspace: op 0/1 dilation/erosion, 2/3 their backward."""
        sv = se_view(se)                         # keeps the SE arrays alive during the call
        return morph_workspace_size(self.handle, make_image(f, L), sv.c, op, make_opts(method, allow_unproven_f32))

    def set_cache_limit(self, nbytes: int):
        """Device-memory budget of the plan cache (least recently used plans are dropped beyond it)."""
        check(morph_ctx_set_cache_limit(self.handle, nbytes), "morph_ctx_set_cache_limit")

    def cache_info(self):
        """(device bytes held by cached plans, number of plans)."""
        return morph_ctx_cache_info(self.handle)

    def plan(self, f, L, se, op=0, method="auto", allow_unproven_f32=False, **_):
        img = make_image(f, L)
        sv = se_view(se)
        return morph_plan_query(self.handle, img, sv.c, op, make_opts(method, allow_unproven_f32))

    # -- batches ---------------------------------------------------------------
    def _problems(self, items):
        """items: (f, L, se, op, out, out_count-or-None) tuples of CUDA tensors."""
        import torch
        keep, probs = [], []
        for (f, L, se, op, out, cnt) in items:
            img = make_image(f, L)
            sv = se_view(se)
            pr = morph_problem()
            pr.f = img
            pr.se = sv.c
            pr.op = 0 if op in (0, "dilate") else 1
            pr.out = out.data_ptr()
            pr.out_count = cnt.data_ptr() if cnt is not None else None
            keep.append(sv)
            probs.append(pr)
        return probs, keep

    def run_batch(self, items, method="auto", stream=None, allow_unproven_f32=False, count_err=None, autotune=False):
        probs, keep = self._problems(items)
        opts = make_opts(method, allow_unproven_f32, count_err is not None, count_err, autotune)
        st = stream if stream is not None else current_stream_handle(self.device)
        check(morph_run_batch(self.handle, probs, opts, st), "morph_run_batch")

    def capture_batch(self, items, method="auto", allow_unproven_f32=False, autotune=False):
        probs, keep = self._problems(items)
        h = morph_batch_capture(self.handle, probs, make_opts(method, allow_unproven_f32, autotune=autotune))
        return CapturedBatch(h, keep)

    def check(self, stream=None):
        st = stream if stream is not None else current_stream_handle(self.device)
        check(morph_stream_check(self.handle, st), "morph_stream_check")

    def launches(self) -> int:
        return morph_launch_count(self.handle)

    def set_wait_limit(self, ns: int):
        """Limit of the kernels' bounded waits (0 = the default 4 s); a failure-handling hook."""
        check(morph_ctx_set_wait_limit(self.handle, ns), "morph_ctx_set_wait_limit")

    def band_work(self) -> int:
        """Multiply-adds of the band-limited contraction the FP8 route needed (synchronises)."""
        return morph_band_work(self.handle)

    def mma_count(self) -> int:
        """tcgen05 MMAs the FP8 direct route issued through this context (synchronises)."""
        return morph_mma_count(self.handle)

    def tc_fp8_peak(self) -> float:
        """TFLOP/s of back-to-back FP8 tcgen05 MMAs on every SM (the tensor pipe's peak)."""
        return morph_tc_fp8_peak(self.handle)

    def profile(self, on: bool):
        check(morph_profile_enable(self.handle, on), "morph_profile_enable")

    def profile_read(self):
        return morph_profile_read(self.handle)


class CapturedBatch:
    """A batch planned once and recorded into a CUDA graph (morph_batch_capture)."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def launch(self, stream=None):
        st = stream if stream is not None else current_stream_handle()
        check(morph_batch_launch(self.handle, st), "morph_batch_launch")

    def close(self):
        if self.handle:
            morph_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_contexts = {}


def get_context(device: int = 0) -> Context:
    with _lock:
        c = _contexts.get(int(device))
    if c is None:
        c = Context(device)
        with _lock:
            _contexts[int(device)] = c
    return c
