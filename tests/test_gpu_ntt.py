"""GPU parity of the exact NTT route (Step 2 modulo a prime > |B|) against
the oracle: bit-exact values and top counts on ragged multi-tile images,
every radix of the transform sizes, 8-bit images with 8-bit offsets (where
the FP32 FFT bound fails), erosion, batches and a full-size configuration on
sampled rows."""
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


def _run(ctx, f, L, se, op, **kw):
    ft = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    fn = ctx.dilate if op == "dilate" else ctx.erode
    out, cnt = fn(ft, L, se, method="ntt", count=True, **kw)
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


# (N, H, W, L, kh, kw, p_in, max_off, origin)
CASES = [
    (1, 37, 53, 16, 7, 7, 0.5, 3, None),          # R = 19 -> Rf = 20 (radix 4 x 5)
    (2, 40, 61, 4, 3, 5, 0.7, 1, (0, 4)),         # R = 5 (radix 5)
    (1, 33, 29, 20, 5, 9, 0.6, 6, (4, 0)),        # R = 26 -> 27 (radix 3^3)
    (3, 17, 17, 32, 9, 9, 1.0, 7, None),
    (1, 25, 70, 256, 5, 3, 0.8, 255, (1, 1)),     # R = 511 -> 512, 8-bit offsets
    (1, 64, 45, 64, 15, 13, 0.5, 7, (3, 12)),
    (1, 300, 290, 256, 41, 37, 0.9, 200, None),   # several tiles, ragged tails
    (1, 9, 300, 2, 1, 1, 1.0, 0, None),           # identity SE, binary image
]


@pytest.mark.parametrize("case", CASES)
def test_random_cases_bit_exact(ctx, case):
    N, H, W, L, kh, kw, p_in, mo, origin = case
    g = wl.rng(hash((N, H, W, L, kh, 17)) & 0xFFFF)
    f = g.integers(0, L, size=(N, H, W)).astype(np.uint8)
    se = wl.se_random(g, kh, kw, p_in, mo, origin=origin)
    for op in ("dilate", "erode"):
        _eq(_run(ctx, f, L, se, op), _ref(f, L, se, op))


@pytest.mark.parametrize("origin", [(-3, 9), (8, -5), (-20, -20), (30, 2)])
def test_origin_outside_the_box(ctx, origin):
    g = wl.rng(hash(origin) & 0xFFFF)
    f = g.integers(0, 64, size=(2, 70, 81)).astype(np.uint8)
    se = wl.se_random(g, 6, 4, 0.5, 5, origin=origin, force_origin=False)
    for op in ("dilate", "erode"):
        _eq(_run(ctx, f, 64, se, op), _ref(f, 64, se, op))


def test_flat_disk(ctx):
    g = wl.rng(91)
    f = g.integers(0, 64, size=(2, 70, 81)).astype(np.uint8)
    disk = wl.se_flat_disk(9)
    _eq(_run(ctx, f, 64, disk, "dilate"), _ref(f, 64, disk, "dilate"))


def test_x1_shape_8bit_large_filter(ctx):
    # the paper's X1 shape at 8 bits (Sec. 4.1): 512 x 512 image, 96 x 96 full-support
    # filter with offsets 0..255 -- where the FP32 FFT cannot be proven exact
    g = wl.rng(92)
    f = g.integers(0, 256, size=(1, 512, 512)).astype(np.uint8)
    se = wl.se_full_random(g, 96, 255)
    info = ctx.plan(torch.from_numpy(f).cuda(), 256, se, method="fft_f64")
    assert not info.f32_bound < 0.5
    got = _run(ctx, f, 256, se, "dilate")
    for rows in [(0, 3), (250, 252), (509, 512)]:
        _eq(got, _ref(f, 256, se, "dilate", rows=rows), rows=rows)


def test_c3_full_size_sampled(ctx):
    p = wl.c3_full_tonal()
    got = _run(ctx, p.f, p.L, p.se, "dilate")
    for rows in [(0, 2), (1500, 1502), (4094, 4096)]:
        _eq(got, _ref(p.f, p.L, p.se, "dilate", rows=rows), rows=rows)


def test_batch_with_ntt_problems(ctx):
    g = wl.rng(93)
    items, refs = [], []
    for (h, w, L, k, mo, op) in [(50, 60, 16, 5, 3, 0), (33, 47, 256, 9, 100, 1), (80, 20, 64, 3, 7, 0)]:
        f = g.integers(0, L, size=(1, h, w)).astype(np.uint8)
        se = wl.se_random(g, k, k, 0.7, mo)
        ft = torch.from_numpy(f).cuda()
        out = torch.empty((1, h, w), dtype=torch.int32, device="cuda")
        cnt = torch.empty_like(out)
        items.append((ft, L, se, op, out, cnt))
        refs.append(_ref(f, L, se, "dilate" if op == 0 else "erode"))
    ctx.run_batch(items, method="ntt")
    ctx.check()
    for it, ref in zip(items, refs):
        _eq((it[4].cpu().numpy(), it[5].cpu().numpy()), ref)


def test_auto_takes_ntt_for_8bit_offsets_and_stays_exact(ctx):
    # 8-bit image and 8-bit offsets with a 64 x 64 filter: the FP32 bound fails, the
    # FP8 route stacks 256 offset levels, and AUTO's estimate favours the NTT
    g = wl.rng(94)
    f = g.integers(0, 256, size=(1, 300, 280)).astype(np.uint8)
    se = wl.se_full_random(g, 64, 255)
    ft = torch.from_numpy(f).cuda()
    assert ctx.plan(ft, 256, se, method="auto").method == 4
    out, cnt = ctx.dilate(ft, 256, se, method="auto", count=True)
    ctx.check()
    for rows in [(0, 3), (140, 143), (297, 300)]:
        _eq((out.cpu().numpy(), cnt.cpu().numpy()), _ref(f, 256, se, "dilate", rows=rows), rows=rows)


def test_plan_cache_stays_within_its_limit(ctx):
    # many distinct SEs: least recently used plans are dropped, results stay exact,
    # and a dropped plan is rebuilt on demand
    g = wl.rng(95)
    f = g.integers(0, 256, size=(1, 120, 130)).astype(np.uint8)
    ft = torch.from_numpy(f).cuda()
    limit = 24 << 20
    ctx.set_cache_limit(limit)
    try:
        ses = [wl.se_full_random(g, 9, 255) for _ in range(12)]
        for se in ses:
            out = ctx.dilate(ft, 256, se, method="ntt")
            ctx.check()
            assert ctx.cache_info()[0] <= limit or ctx.cache_info()[1] == 1
            assert np.array_equal(out.cpu().numpy(), _ref(f, 256, se, "dilate")[0])
        out = ctx.dilate(ft, 256, ses[0], method="ntt")
        ctx.check()
        assert np.array_equal(out.cpu().numpy(), _ref(f, 256, ses[0], "dilate")[0])
    finally:
        ctx.set_cache_limit(16 << 30)
