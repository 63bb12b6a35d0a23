"""Host-side planning through the C ABI, without a GPU: morph_workspace_size
with a NULL context runs the validation, the route choice (AUTO's fitted
time models), the FP8, FFT and NTT tilings and the backward chunking on the
host only.  Image data pointers are never dereferenced on this path."""
import ctypes

import numpy as np
import pytest

from paper_2305_03018_gb300 import morph as M
from paper_2305_03018_gb300 import workloads as wl

pytestmark = pytest.mark.timeout(60)
_DUMMY = ctypes.create_string_buffer(16)


def _img(n, h, w, L, dtype=M.MORPH_U8):
    im = M.morph_image()
    im.data = ctypes.addressof(_DUMMY)
    im.dtype = dtype
    im.n, im.h, im.w = n, h, w
    im.row_stride = w
    im.batch_stride = h * w
    im.L = L
    return im


def _ws(im, se, op, method="auto"):
    sv = M.se_view(se)
    return M.morph_workspace_size(None, im, sv.c, op, M.make_opts(method))


def _band_bytes(n, h, w):
    # one (hi, lb) int pair per 16 image rows (two at least: a 64-row unit has two 32-row slabs)
    # by 16 columns, 256-byte rounded, then 256 bytes for the launch's unit counter
    return -(-n * max(-(-h // 16), 2) * -(-w // 16) * 8 // 256) * 256 + 256


def test_direct_and_backward_sizes_follow_their_layouts(bwd_chunks):
    g = wl.rng(61)
    se = wl.se_random(g, 9, 7, 0.6, 5)
    im = _img(2, 200, 300, 64)
    # indicator planes: n h L round32(w + 31) bytes (room for the column shift that aligns K windows),
    # then the per-unit grey-level bands
    assert _ws(im, se, 0, "direct_fp8") == _ws(im, se, 1, "direct_fp8") == 2 * 200 * 64 * 352 + _band_bytes(2, 200, 300)
    # backward: a float share per pixel (256-byte rounded) + a partial sum per (tap, chunk)
    ntaps = int(np.count_nonzero(se.mask))
    exp = -(-2 * 200 * 300 * 4 // 256) * 256 + ntaps * bwd_chunks(2, 200, 300, ntaps) * 4
    assert _ws(im, se, 2) == _ws(im, se, 3) == exp
    # more than 1024 taps: the pixel-chunked gather's layout
    big = wl.se_full_random(g, 33, 3)
    exp = -(-2 * 200 * 300 * 4 // 256) * 256 + 33 * 33 * bwd_chunks(2, 200, 300, 33 * 33) * 4
    assert _ws(im, big, 2) == exp



def test_transform_routes_plan_on_the_host():
    g = wl.rng(62)
    for (n, L, k, mo) in [(512, 256, 64, 255), (2048, 16, 204, 15), (300, 64, 31, 4), (64, 2, 3, 0)]:
        se = wl.se_full_random(g, k, mo)
        im = _img(1, n, n, L)
        ntt = _ws(im, se, 0, "ntt")
        f64 = _ws(im, se, 0, "fft_f64")
        assert ntt > 0 and f64 > 0
        sizes = {ntt, f64, _ws(im, se, 0, "direct_fp8")}
        try:
            sizes.add(_ws(im, se, 0, "fft_f32"))
        except M.MorphError as e:                  # FP32 refused where its bound fails
            assert e.status == M.MORPH_E_PRECISION
        assert _ws(im, se, 0, "auto") in sizes


def test_auto_prefers_ntt_for_8bit_offsets_and_fp8_for_small_flat():
    g = wl.rng(63)
    big = wl.se_full_random(g, 96, 255)
    im = _img(1, 512, 512, 256)
    assert _ws(im, big, 0, "auto") == _ws(im, big, 0, "ntt")
    small = wl.se_flat_square(3)
    im2 = _img(1, 1024, 1024, 16)
    assert _ws(im2, small, 0, "auto") == _ws(im2, small, 0, "direct_fp8")


def test_invalid_requests_are_refused():
    se = wl.se_flat_square(3)
    sv = M.se_view(se)
    bytes_ = ctypes.c_size_t(0)
    lib = M.load_library()
    im = _img(1, 10, 10, 16)
    assert lib.morph_workspace_size(None, ctypes.byref(im), ctypes.byref(sv.c), 4, None, ctypes.byref(bytes_)) \
        == M.MORPH_E_INVAL
    bad = _img(1, 10, 10, 1)                       # L < 2
    assert lib.morph_workspace_size(None, ctypes.byref(bad), ctypes.byref(sv.c), 0, None, ctypes.byref(bytes_)) \
        == M.MORPH_E_INVAL
    assert lib.morph_workspace_size(None, ctypes.byref(im), ctypes.byref(sv.c), 0, None, None) == M.MORPH_E_INVAL


def test_huge_offsets_plan_only_the_fp8_route():
    m = np.ones((3, 3), np.uint8)
    o = np.array([[0, 65535, 7], [3, 0, 40000], [1, 2, 3]], np.int32)
    se = wl.SE(m, o, (1, 1), "huge")
    im = _img(1, 64, 64, 256)
    assert _ws(im, se, 0, "auto") == _ws(im, se, 0, "direct_fp8") == 64 * 256 * 96 + _band_bytes(1, 64, 64)
    for method in ("ntt", "fft_f64"):
        with pytest.raises(M.MorphError) as ei:
            _ws(im, se, 0, method)
        assert ei.value.status == M.MORPH_E_UNSUPPORTED


def _direct_info(shape, L, se):
    sv = M.se_view(se)
    return M.morph_plan_query(None, _img(*shape, L), sv.c, 0, M.make_opts("direct_fp8"))


def test_chunk_width_follows_the_plan_rules():
    g = wl.rng(71)
    # 16 < L <= 64, a large SE on a 2048^2 image: 4-level chunks of 64-row units
    info = _direct_info((1, 2048, 2048), 64, wl.se_flat_disk(31))
    assert (info.tile_h, info.level_chunks) == (64, 16)
    # the same SE on a small image (fewer than two waves of 64-row units): 8-level chunks
    info = _direct_info((1, 300, 300), 64, wl.se_flat_disk(31))
    assert (info.tile_h, info.level_chunks) == (32, 8)
    # a small SE (few MMAs per accumulation): 8-level chunks
    info = _direct_info((1, 2048, 2048), 64, wl.se_full_random(g, 9, 7))
    assert (info.tile_h, info.level_chunks) == (32, 8)
    # offsets beyond 4095 - L: the packed running results could not hold the degrees
    m = np.ones((31, 31), np.uint8)
    off = (g.integers(0, 2, size=m.shape) * 5000).astype(np.int32)
    info = _direct_info((1, 2048, 2048), 64, wl.SE(m, off, (15, 15), "far"))
    assert (info.tile_h, info.level_chunks) == (32, 8)
    # L <= 16 and L > 64: 16-level chunks of 16-row units
    for L in (16, 256):
        info = _direct_info((1, 2048, 2048), L, wl.se_flat_disk(31))
        assert (info.tile_h, info.level_chunks) == (16, -(-L // 16))
