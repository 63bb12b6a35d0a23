"""GPU parity of the FP8 tensor-core route (Steps 1-3) against the CPU oracle.

Every comparison is bit-exact: the dilation/erosion value and the top count
(the number of taps attaining it) at every pixel, or at sampled rows where
the oracle would take too long.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2305_03018_gb300 import workloads as wl
from tests.conftest import GOLDEN

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2305_03018_gb300.morph import get_context
    assert torch.cuda.is_available()
    return get_context(0)


def _run(ctx, f_np, L, se, op="dilate", method="direct_fp8", dtype=None):
    ft = torch.from_numpy(np.ascontiguousarray(f_np if dtype is None else f_np.astype(dtype))).cuda()
    fn = ctx.dilate if op == "dilate" else ctx.erode
    out, cnt = fn(ft, L, se, method=method, count=True)
    ctx.check()
    return out.cpu().numpy(), cnt.cpu().numpy()


def _ref(f_np, L, se, op="dilate", rows=None):
    fn = oracle.dilate if op == "dilate" else oracle.erode
    return fn(f_np, L, se.mask, se.offset, se.origin, rows=rows, nthreads=0)


def _assert_equal(got, ref, rows=None):
    gD, gC = got
    rD, rC = ref
    if rows is not None:
        sl = (slice(None), slice(rows[0], rows[1]))
        gD, gC, rD, rC = gD[sl], gC[sl], rD[sl], rC[sl]
    bad = np.argwhere(gD != rD)
    assert bad.size == 0, f"{len(bad)} value mismatches, first at {bad[:5].tolist()}: got {gD[tuple(bad[0])]} want {rD[tuple(bad[0])]}"
    bad = np.argwhere(gC != rC)
    assert bad.size == 0, f"{len(bad)} count mismatches, first at {bad[:5].tolist()}"


def test_paper_example_on_gpu(ctx):
    with open(os.path.join(GOLDEN, "example2_5.json")) as fh:
        ex = json.load(fh)
    f = np.array(ex["image"], np.uint8)[None, None, :]
    flt = ex["filter"]
    se = wl.SE(np.array([[0 if v is None else 1 for v in flt]], np.uint8),
               np.array([[0 if v is None else v for v in flt]], np.int32), (0, ex["filter_origin"]))
    D, cD = _run(ctx, f, ex["L"], se)
    assert D.ravel().tolist() == ex["dilation"]
    assert cD.ravel().tolist() == [1] * 6


CASES = [
    # (N, H, W, L, kh, kw, p_in, max_off, origin)
    (1, 37, 53, 16, 7, 7, 0.5, 3, None),
    (2, 64, 200, 2, 3, 5, 0.7, 0, (0, 4)),
    (1, 33, 129, 20, 5, 9, 0.6, 6, (4, 0)),
    (3, 17, 17, 32, 9, 9, 1.0, 7, None),
    (1, 40, 300, 64, 15, 15, 0.5, 7, (2, 13)),
    (1, 24, 70, 100, 4, 6, 0.8, 30, (1, 2)),
    (1, 19, 150, 256, 11, 13, 0.4, 15, None),
    (1, 9, 31, 256, 3, 3, 1.0, 200, None),       # 9 offset levels -> 2 passes at G = 8? large R
    (1, 50, 45, 16, 1, 1, 1.0, 0, None),
    (1, 30, 40, 64, 31, 31, 0.5, 20, None),      # > 8 levels: several passes
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_random_cases_bit_exact(ctx, case, op):
    N, H, W, L, kh, kw, p_in, mo, origin = case
    g = wl.rng(hash((N, H, W, L, kh, kw, mo)) & 0xFFFF)
    f = g.integers(0, L, size=(N, H, W)).astype(np.uint8 if L <= 256 else np.int32)
    se = wl.se_random(g, kh, kw, p_in, mo, origin=origin)
    _assert_equal(_run(ctx, f, L, se, op), _ref(f, L, se, op))


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.int32])
def test_input_dtypes(ctx, dtype):
    g = wl.rng(11)
    f = g.integers(0, 64, size=(2, 21, 47))
    se = wl.se_random(g, 5, 5, 0.6, 3)
    _assert_equal(_run(ctx, f, 64, se, dtype=dtype), _ref(f.astype(np.int32), 64, se))


def test_strided_view(ctx):
    g = wl.rng(12)
    base = g.integers(0, 16, size=(3, 40, 90)).astype(np.uint8)
    ft = torch.from_numpy(base).cuda()[:, 5:35, 7:80]           # non-contiguous rows
    se = wl.se_random(g, 7, 5, 0.5, 2)
    D, cD = ctx.dilate(ft, 16, se, method="direct_fp8", count=True)
    ctx.check()
    ref = _ref(np.ascontiguousarray(base[:, 5:35, 7:80]), 16, se)
    _assert_equal((D.cpu().numpy(), cD.cpu().numpy()), ref)


def test_edge_shapes(ctx):
    g = wl.rng(13)
    # 1x1 image; SE larger than the image; origin outside the support / box
    for (H, W, kh, kw, origin) in [(1, 1, 3, 3, (1, 1)), (2, 3, 9, 11, (8, 0)), (5, 4, 7, 7, (-2, 9)),
                                   (1, 200, 1, 63, (0, 31)), (200, 1, 63, 1, (31, 0))]:
        f = g.integers(0, 16, size=(1, H, W)).astype(np.uint8)
        se = wl.se_random(g, kh, kw, 0.5, 3, origin=origin, force_origin=False)
        if se.taps == 0:
            se.mask[0, 0] = 1
        for op in ("dilate", "erode"):
            _assert_equal(_run(ctx, f, 16, se, op), _ref(f, 16, se, op))


def test_empty_support(ctx):
    f = np.arange(60, dtype=np.uint8).reshape(1, 6, 10) % 16
    se = wl.SE(np.zeros((3, 3), np.uint8), np.zeros((3, 3), np.int32), (1, 1))
    for op in ("dilate", "erode"):
        _assert_equal(_run(ctx, f, 16, se, op), _ref(f, 16, se, op))


def test_max_count_63x63_flat(ctx):
    # constant image, full 63x63 flat SE: the top count reaches 3969 in the interior
    f = np.full((1, 100, 130), 9, np.uint8)
    se = wl.se_flat_square(63)
    D, cD = _run(ctx, f, 16, se)
    assert (D == 9).all()
    assert cD.max() == 3969
    _assert_equal((D, cD), _ref(f, 16, se))


def test_c1_full_config(ctx):
    p = wl.c1_small_dilation()
    for op in ("dilate", "erode"):
        _assert_equal(_run(ctx, p.f, p.L, p.se, op), _ref(p.f, p.L, p.se, op))


@pytest.mark.parametrize("which", [0, 2])
def test_c2_full_size_sampled_rows(ctx, which):
    probs = wl.c2_large_filter()
    for p in probs[which:which + 2]:           # dilation and erosion of one SE
        got = _run(ctx, p.f, p.L, p.se, p.op)
        for rows in [(0, 3), (1020, 1023), (2045, 2048)]:
            _assert_equal(got, _ref(p.f, p.L, p.se, p.op, rows=rows), rows=rows)


def test_data_error_reported(ctx):
    from paper_2305_03018_gb300.morph import MORPH_E_RANGE, MorphError
    f = np.zeros((1, 8, 8), np.uint8)
    f[0, 3, 3] = 40
    ft = torch.from_numpy(f).cuda()
    ctx.dilate(ft, 32, wl.se_flat_square(3), method="direct_fp8")
    with pytest.raises(MorphError) as ei:
        ctx.check()
    assert ei.value.status == MORPH_E_RANGE
    ctx.check()                                  # the error word was cleared


def test_workspace_size_matches_plan_and_is_host_only(bwd_chunks):
    from paper_2305_03018_gb300.morph import get_context
    ctx = get_context(0)
    g = wl.rng(61)
    f = torch.from_numpy(g.integers(0, 64, size=(2, 200, 300)).astype(np.uint8)).cuda()
    se = wl.se_random(g, 9, 7, 0.6, 5)
    for method in ("direct_fp8", "fft_f64", "ntt", "auto"):
        for op in (0, 1):
            ws = ctx.workspace_size(f, 64, se, op=op, method=method)
            assert ws == ctx.plan(f, 64, se, op=op, method=method).workspace_bytes, (method, op)
    # planes n h L round32(w + 31), then one (hi, lb) pair per 16 image rows x 16 columns and the
    # launch's unit counter
    band = -(-2 * 13 * 19 * 8 // 256) * 256 + 256
    assert ctx.workspace_size(f, 64, se, op=0, method="direct_fp8") == 2 * 200 * 64 * 352 + band
    # backward: one float share per pixel (rounded to 256 B) plus one partial sum per (tap, chunk)
    ntaps = int(np.count_nonzero(se.mask))
    exp = ((2 * 200 * 300 * 4 + 255) // 256) * 256 + ntaps * bwd_chunks(2, 200, 300, ntaps) * 4
    assert ctx.workspace_size(f, 64, se, op=2) == exp == ctx.workspace_size(f, 64, se, op=3)


def test_huge_sparse_offsets():
    # offsets up to 65535 (R = L + 65535): only the FP8 route applies (its offset
    # levels are the distinct offsets); the transform routes refuse the size
    from paper_2305_03018_gb300.morph import MORPH_E_UNSUPPORTED, MorphError, get_context
    ctx = get_context(0)
    g = wl.rng(64)
    f = g.integers(0, 256, size=(1, 70, 90)).astype(np.uint8)
    m = (g.random((7, 9)) < 0.6).astype(np.uint8)
    m[3, 4] = 1
    o = (g.choice([0, 1000, 40000, 65535], size=m.shape) * m).astype(np.int32)
    se = wl.SE(m, o, (3, 4), "huge")
    ft = torch.from_numpy(f).cuda()
    for op in ("dilate", "erode"):
        fn = ctx.dilate if op == "dilate" else ctx.erode
        out, cnt = fn(ft, 256, se, method="auto", count=True)
        ctx.check()
        ref = (oracle.dilate if op == "dilate" else oracle.erode)(f, 256, m, o, (3, 4))
        assert np.array_equal(out.cpu().numpy(), ref[0]) and np.array_equal(cnt.cpu().numpy(), ref[1])
    for method in ("ntt", "fft_f64"):
        with pytest.raises(MorphError) as ei:
            ctx.dilate(ft, 256, se, method=method)
        assert ei.value.status == MORPH_E_UNSUPPORTED
