"""Full-size configurations on the GPU against the oracle, every pixel: the
value and the top count of each output pixel (the method is exact, Sec. 4.3
reports a mean absolute error of 0).  The oracle runs on all host cores; each
reference is computed once per module."""
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


@pytest.fixture(scope="module")
def c3():
    p = wl.c3_full_tonal()
    ref = oracle.dilate(p.f, p.L, p.se.mask, p.se.offset, p.se.origin, nthreads=0)
    return p, ref


@pytest.fixture(scope="module")
def c2():
    probs = wl.c2_large_filter()
    refs = []
    for p in probs:
        fn = oracle.dilate if p.op == "dilate" else oracle.erode
        refs.append(fn(p.f, p.L, p.se.mask, p.se.offset, p.se.origin, nthreads=0))
    return probs, refs


def _same(got, ref, what):
    D, cD = (t.cpu().numpy() for t in got)
    rD, rC = ref
    bad = np.argwhere(D != rD)
    assert bad.size == 0, (what, "values differ", len(bad), bad[:5].tolist())
    bad = np.argwhere(cD != rC)
    assert bad.size == 0, (what, "top counts differ", len(bad), bad[:5].tolist())


@pytest.mark.parametrize("method", ["direct_fp8", "ntt", "fft_f32", "auto"])
def test_c3_full_tonal_range_every_pixel(ctx, c3, method):
    p, ref = c3
    ft = torch.from_numpy(p.f).cuda()
    err = torch.zeros(1, dtype=torch.float32, device="cuda")
    kw = {"count_err": err} if method == "fft_f32" else {}
    got = ctx.dilate(ft, p.L, p.se, method=method, count=True, **kw)
    ctx.check()
    _same(got, ref, f"C3 {method}")
    if method == "fft_f32":
        info = ctx.plan(ft, p.L, p.se, method="fft_f32")
        assert info.f32_bound < 0.5
        assert 0.0 <= float(err.item()) <= info.f32_bound


@pytest.mark.parametrize("method", ["direct_fp8", "ntt"])
def test_c2_every_operation_every_pixel(ctx, c2, method):
    probs, refs = c2
    ft = torch.from_numpy(probs[0].f).cuda()
    for p, ref in zip(probs, refs):
        fn = ctx.dilate if p.op == "dilate" else ctx.erode
        got = fn(ft, p.L, p.se, method=method, count=True)
        ctx.check()
        _same(got, ref, f"{p.name} {method}")


def test_c2_fp64_fft_every_pixel(ctx, c2):
    probs, refs = c2
    p, ref = probs[2], refs[2]                  # 63x63 non-flat dilation
    ft = torch.from_numpy(p.f).cuda()
    got = ctx.dilate(ft, p.L, p.se, method="fft_f64", count=True)
    ctx.check()
    _same(got, ref, "C2 63x63 fft_f64")


@pytest.mark.parametrize("shape,L,k", [((1, 8192, 8192), 16, 5), ((1, 16, 70000), 64, 7), ((3, 2500, 40), 256, 9)])
def test_large_and_extreme_shapes_every_pixel(ctx, shape, L, k):
    # a 67 Mpix image, a very wide strip and tall narrow images through AUTO
    g = wl.rng(sum(shape) + L)
    f = g.integers(0, L, size=shape).astype(np.uint8)
    se = wl.se_random(g, k, k, 0.6, max(1, L // 16))
    ft = torch.from_numpy(f).cuda()
    got = ctx.dilate(ft, L, se, method="auto", count=True)
    ctx.check()
    ref = oracle.dilate(f, L, se.mask, se.offset, se.origin, nthreads=0)
    _same(got, ref, f"extreme {shape}")
