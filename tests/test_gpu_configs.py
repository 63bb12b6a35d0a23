"""Full-size configurations on the GPU, checked on sampled rows against the
oracle (the whole image would take the oracle minutes)."""
import numpy as np
import pytest

import oracle
from paper_2305_03018_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROWS = [(0, 2), (1500, 1502), (4094, 4096)]


@pytest.fixture(scope="module")
def ctx():
    from paper_2305_03018_gb300.morph import get_context
    return get_context(0)


@pytest.fixture(scope="module")
def c3():
    return wl.c3_full_tonal()


def _sampled(p, got, rows_list):
    D, cD = got
    for rows in rows_list:
        rD, rC = oracle.dilate(p.f, p.L, p.se.mask, p.se.offset, p.se.origin, rows=rows, nthreads=0)
        sl = (slice(None), slice(*rows))
        assert np.array_equal(D[sl], rD[sl]), rows
        assert np.array_equal(cD[sl], rC[sl]), rows


@pytest.mark.parametrize("method", ["direct_fp8", "fft_f32"])
def test_c3_full_tonal_range(ctx, c3, method):
    ft = torch.from_numpy(c3.f).cuda()
    err = torch.zeros(1, dtype=torch.float32, device="cuda")
    kw = {"count_err": err} if method == "fft_f32" else {}
    D, cD = ctx.dilate(ft, c3.L, c3.se, method=method, count=True, **kw)
    ctx.check()
    _sampled(c3, (D.cpu().numpy(), cD.cpu().numpy()), ROWS)
    if method == "fft_f32":
        info = ctx.plan(ft, c3.L, c3.se, method="fft_f32")
        assert info.f32_bound < 0.5
        assert 0.0 <= float(err.item()) <= info.f32_bound


def test_c2_fp64_fft_sampled(ctx):
    p = wl.c2_large_filter()[2]                  # 63x63 non-flat dilation
    ft = torch.from_numpy(p.f).cuda()
    D, cD = ctx.dilate(ft, p.L, p.se, method="fft_f64", count=True)
    ctx.check()
    _sampled(p, (D.cpu().numpy(), cD.cpu().numpy()), [(0, 2), (2046, 2048)])


@pytest.mark.parametrize("shape,L,k", [((1, 8192, 8192), 16, 5), ((1, 16, 70000), 64, 7), ((3, 2500, 40), 256, 9)])
def test_large_and_extreme_shapes_sampled(ctx, shape, L, k):
    # a 67 Mpix image, a very wide strip and tall narrow images through AUTO, checked on sampled rows
    g = wl.rng(sum(shape) + L)
    f = g.integers(0, L, size=shape).astype(np.uint8)
    se = wl.se_random(g, k, k, 0.6, max(1, L // 16))
    ft = torch.from_numpy(f).cuda()
    D, cD = ctx.dilate(ft, L, se, method="auto", count=True)
    ctx.check()
    H = shape[1]
    rows = [(0, 2), (H // 2, H // 2 + 1), (H - 2, H)] if H > 4 else [(0, H)]
    p = wl.Problem(f, L, se, "dilate", "extreme")
    _sampled(p, (D.cpu().numpy(), cD.cpu().numpy()), rows)
