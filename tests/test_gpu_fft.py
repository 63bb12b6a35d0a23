"""GPU parity of the FFT routes (FP64 and FP32 Step 2) against the oracle.

FP32 runs only where its a-priori round-off bound proves the counts exact
(< 0.5), unless the caller opts in; the measured max |C - rint C| is checked
against that bound.
"""
import numpy as np
import pytest

import oracle
from paper_2305_03018_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2305_03018_gb300.morph import get_context
    return get_context(0)


def _run(ctx, f, L, se, op, method, **kw):
    ft = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    fn = ctx.dilate if op == "dilate" else ctx.erode
    out, cnt = fn(ft, L, se, method=method, count=True, **kw)
    ctx.check()
    return out.cpu().numpy(), cnt.cpu().numpy()


def _ref(f, L, se, op, rows=None):
    fn = oracle.dilate if op == "dilate" else oracle.erode
    return fn(f, L, se.mask, se.offset, se.origin, rows=rows, nthreads=0)


def _eq(got, ref, rows=None):
    for a, b in zip(got, ref):
        if rows is not None:
            a, b = a[:, rows[0]:rows[1]], b[:, rows[0]:rows[1]]
        bad = np.argwhere(a != b)
        assert bad.size == 0, f"{len(bad)} mismatches, first {bad[:3].tolist()}"


CASES = [
    (1, 37, 53, 16, 7, 7, 0.5, 3, None),
    (2, 40, 61, 4, 3, 5, 0.7, 1, (0, 4)),
    (1, 33, 29, 20, 5, 9, 0.6, 6, (4, 0)),
    (3, 17, 17, 32, 9, 9, 1.0, 7, None),
    (1, 25, 70, 256, 5, 3, 0.8, 15, (1, 1)),
    (1, 64, 45, 64, 15, 13, 0.5, 7, (3, 12)),
]


@pytest.mark.parametrize("method", ["fft_f64", "fft_f32"])
@pytest.mark.parametrize("case", CASES)
def test_random_cases_bit_exact(ctx, method, case):
    N, H, W, L, kh, kw, p_in, mo, origin = case
    g = wl.rng(hash((N, H, W, L, kh)) & 0xFFFF)
    f = g.integers(0, L, size=(N, H, W)).astype(np.uint8)
    se = wl.se_random(g, kh, kw, p_in, mo, origin=origin)
    for op in ("dilate", "erode"):
        _eq(_run(ctx, f, L, se, op, method), _ref(f, L, se, op))


def test_c1_fp64_and_fp32_with_measured_error(ctx):
    p = wl.c1_small_dilation()
    ft = torch.from_numpy(p.f).cuda()
    info = ctx.plan(ft, p.L, p.se, method="fft_f32")
    assert info.f32_bound < 0.5 and info.f64_bound < 1e-6
    ref = _ref(p.f, p.L, p.se, "dilate")
    for method, lim in (("fft_f64", info.f64_bound), ("fft_f32", info.f32_bound)):
        err = torch.zeros(1, dtype=torch.float32, device="cuda")
        got = _run(ctx, p.f, p.L, p.se, "dilate", method, count_err=err)
        _eq(got, ref)
        e = float(err.item())
        assert 0.0 <= e <= lim, (method, e, lim)


def test_fp32_refused_where_bound_fails_and_opt_in_runs(ctx):
    from paper_2305_03018_gb300.morph import MORPH_E_PRECISION, MorphError
    g = wl.rng(77)
    f = g.integers(0, 64, size=(1, 300, 260)).astype(np.uint8)
    se = wl.se_full_random(g, 63, 7)
    ft = torch.from_numpy(f).cuda()
    info = ctx.plan(ft, 64, se, method="fft_f64")
    assert info.f32_bound > 0.5
    with pytest.raises(MorphError) as ei:
        ctx.dilate(ft, 64, se, method="fft_f32")
    assert ei.value.status == MORPH_E_PRECISION
    err = torch.zeros(1, dtype=torch.float32, device="cuda")
    got = _run(ctx, f, 64, se, "dilate", "fft_f32", allow_unproven_f32=True, count_err=err)
    rows = (120, 126)
    _eq(got, _ref(f, 64, se, "dilate", rows=rows), rows=rows)
    assert float(err.item()) < 0.5


def test_multi_tile_fp64(ctx):
    # wider than one 2048-point transform: several overlap-save tiles per row
    g = wl.rng(78)
    f = g.integers(0, 16, size=(1, 40, 2300)).astype(np.uint8)
    se = wl.se_random(g, 5, 31, 0.5, 3, origin=(2, 3))
    for op in ("dilate", "erode"):
        _eq(_run(ctx, f, 16, se, op, "fft_f64"), _ref(f, 16, se, op))


def test_fp32_tiles_shrink_to_meet_bound(ctx):
    # L = 256 with a 25x25 full SE (625 taps): one 300x310 tile would break the
    # FP32 bound, so the planner must pick smaller tiles
    g = wl.rng(79)
    f = g.integers(0, 256, size=(1, 300, 310)).astype(np.uint8)
    se = wl.se_full_random(g, 25, 15)
    ft = torch.from_numpy(f).cuda()
    info = ctx.plan(ft, 256, se, method="fft_f32")
    assert info.method == 2 and info.tile_w < 310 and info.tile_h < 300
    err = torch.zeros(1, dtype=torch.float32, device="cuda")
    _eq(_run(ctx, f, 256, se, "dilate", "fft_f32", count_err=err), _ref(f, 256, se, "dilate"))
    assert float(err.item()) < 0.5


def test_auto_route_is_exact(ctx):
    for p in [wl.c1_small_dilation()]:
        _eq(_run(ctx, p.f, p.L, p.se, "dilate", "auto"), _ref(p.f, p.L, p.se, "dilate"))


@pytest.mark.parametrize("method", ["fft_f64", "fft_f32"])
@pytest.mark.parametrize("origin", [(-3, 9), (8, -5), (-20, -20), (30, 2)])
def test_origin_outside_the_box(ctx, method, origin):
    # the output's torus position (q + reach) mod N wraps when the origin lies outside the SE box
    g = wl.rng(hash(origin) & 0xFFFF)
    f = g.integers(0, 32, size=(2, 70, 81)).astype(np.uint8)
    se = wl.se_random(g, 6, 4, 0.6, 4, origin=origin, force_origin=False)
    for op in ("dilate", "erode"):
        _eq(_run(ctx, f, 32, se, op, method), _ref(f, 32, se, op))


def test_fp64_long_column_axis(ctx):
    # a 2048^2 image with a 204^2 full filter plans column transforms longer than 1163 points:
    # the SE spectrum's column pass then no longer fits four columns per CTA in shared memory
    g = wl.rng(2048 + 204 + 4)
    f = g.integers(0, 16, size=(1, 2048, 2048)).astype(np.uint8)
    se = wl.se_full_random(g, 204, 15)
    info = ctx.plan(torch.from_numpy(f).cuda(), 16, se, method="fft_f64")
    assert info.fft_ny * 16 * 11 > 200 * 1024, info.fft_ny
    rows = (1000, 1002)
    _eq(_run(ctx, f, 16, se, "dilate", "fft_f64"), _ref(f, 16, se, "dilate", rows=rows), rows=rows)
