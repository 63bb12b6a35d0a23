"""The FP8 route's per-unit grey-level bands against the oracle.

The direct kernel contracts, for each unit of output pixels, only the grey
levels that can hold a top degree: from a lower bound on the unit's smallest
dilation value (a max over a subset of the taps) minus max b, up to the
largest level in the unit's input window.  These inputs make that band wide,
empty of useful levels, or the lower bound absent, and every result must stay
bit-exact (values and top counts).  The MMA counter shows the band at work.
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


def _both_ops(ctx, f, L, se, method="direct_fp8"):
    ft = torch.from_numpy(f).cuda()
    for op in ("dilate", "erode"):
        fn = ctx.dilate if op == "dilate" else ctx.erode
        D, cD = fn(ft, L, se, method=method, count=True)
        ctx.check()
        ofn = oracle.dilate if op == "dilate" else oracle.erode
        rD, rC = ofn(f, L, se.mask, se.offset, se.origin, nthreads=0)
        assert np.array_equal(D.cpu().numpy(), rD), (op, se.name)
        assert np.array_equal(cD.cpu().numpy(), rC), (op, se.name)


def test_wide_offsets_make_many_chunks():
    # offsets up to 255 at L = 256: the band reaches down max b levels below the lower bound
    from paper_2305_03018_gb300.morph import get_context
    g = wl.rng(801)
    f = g.integers(0, 256, size=(1, 150, 170)).astype(np.uint8)
    _both_ops(get_context(0), f, 256, wl.se_random(g, 11, 13, 0.5, 255, origin=(5, 6)))


def test_sparse_bright_pixels_on_a_dark_image(ctx):
    # windows that hold one bright pixel while most pixels of the unit see only dark ones:
    # hi = L - 1 with a low lower bound, so a unit spans every chunk
    g = wl.rng(802)
    for L in (64, 256):
        f = np.zeros((2, 130, 190), np.uint8)
        idx = g.integers(0, f.size, size=40)
        f.reshape(-1)[idx] = L - 1
        f.reshape(-1)[g.integers(0, f.size, size=40)] = L // 2
        for se in (wl.se_flat_disk(9), wl.se_random(g, 9, 9, 0.4, 3, origin=(1, 7))):
            _both_ops(ctx, f, L, se)


def test_constant_and_two_level_images(ctx):
    g = wl.rng(803)
    for L, val in ((16, 0), (64, 63), (256, 200)):
        f = np.full((1, 77, 140), val, np.uint8)
        _both_ops(ctx, f, L, wl.se_full_random(g, 7, 2))
    f = (g.integers(0, 2, size=(1, 120, 120)) * 255).astype(np.uint8)   # checkerboard-like 0 / 255
    _both_ops(ctx, f, 256, wl.se_random(g, 15, 15, 0.3, 9))


def test_origin_outside_the_support_and_the_box(ctx):
    # no tap of the lower-bound subset is valid near some borders: those units keep every level
    g = wl.rng(804)
    f = g.integers(0, 64, size=(1, 90, 110)).astype(np.uint8)
    m = np.zeros((5, 5), np.uint8)
    m[0, 0] = m[4, 4] = m[0, 4] = 1
    se = wl.SE(m, g.integers(0, 5, size=(5, 5)).astype(np.int32) * m, (2, 2), "corners")
    _both_ops(ctx, f, 64, se)
    far = wl.se_random(g, 7, 5, 0.6, 4, origin=(-9, 12), force_origin=False)
    _both_ops(ctx, f, 64, far)


def test_smooth_image_bands_in_a_batch(ctx):
    # smooth 8-bit content: narrow bands that differ from unit to unit, in one batched launch
    g = wl.rng(805)
    img = wl.gauss_blurred_u8(g, 256, 4.0)
    probs = []
    for k, (op, se) in enumerate([("dilate", wl.se_random_convex(g, 31, 12, 15)),
                                  ("erode", wl.se_random_convex(g, 21, 12, 7)),
                                  ("dilate", wl.se_flat_disk(12)),
                                  ("erode", wl.se_full_random(g, 9, 30))]):
        probs.append(wl.Problem(img[None, 17 * k:17 * k + 200, :230].copy(), 256, se, op, f"s{k}"))
    items, outs = [], []
    for p in probs:
        ft = torch.from_numpy(p.f).cuda()
        o = torch.full(ft.shape, -9, dtype=torch.int32, device="cuda")
        c = torch.full(ft.shape, -9, dtype=torch.int32, device="cuda")
        items.append((ft, p.L, p.se, p.op, o, c))
        outs.append((o, c))
    ctx.run_batch(items, method="direct_fp8")
    ctx.check()
    for p, (o, c) in zip(probs, outs):
        fn = oracle.dilate if p.op == "dilate" else oracle.erode
        rD, rC = fn(p.f, p.L, p.se.mask, p.se.offset, p.se.origin, nthreads=0)
        assert np.array_equal(o.cpu().numpy(), rD), p.name
        assert np.array_equal(c.cpu().numpy(), rC), p.name


def test_constant_image_issues_one_chunk_per_unit(ctx):
    # flat SE on a constant image: lower bound = top = the constant, so each unit contracts
    # one chunk of levels instead of all L / Lc chunks
    L = 256
    f = torch.full((1, 256, 512), 77, dtype=torch.uint8, device="cuda")
    se = wl.se_flat_disk(7)
    info = ctx.plan(f, L, se, method="direct_fp8")
    full = info.est_flop / (2.0 * 128 * 256 * 32)         # MMAs with every level
    m0, w0 = ctx.mma_count(), ctx.band_work()
    D, cD = ctx.dilate(f, L, se, method="direct_fp8", count=True)
    issued = ctx.mma_count() - m0
    work = ctx.band_work() - w0
    ctx.check()
    assert issued * info.level_chunks == full
    assert int(D.min()) == int(D.max()) == 77
    # the band-limited work: every unit's band is the single level 77, so each pixel needs |B|
    # multiply-adds
    assert work == se.taps * 256 * 512


def test_four_level_chunks_of_64_row_units(ctx):
    # 16 < L <= 64 with enough MMAs per accumulation and two waves of units: 64-row units whose
    # levels come in chunks of 4 and whose running results are packed; ragged bottom and right
    # edges, a unit whose second 32-row slab lies below the image, dilation and erosion
    g = wl.rng(806)
    f = g.integers(0, 64, size=(1, 1100, 2100)).astype(np.uint8)
    for se in (wl.se_flat_disk(15), wl.se_random(g, 31, 31, 0.7, 7, origin=(3, 17))):
        info = ctx.plan(torch.from_numpy(f).cuda(), 64, se, method="direct_fp8")
        assert (info.tile_h, info.level_chunks) == (64, 16), se.name
        _both_ops(ctx, f, 64, se)


def test_batch_mixes_chunk_widths(ctx):
    # one band launch and one persistent direct launch over problems with 4-, 8- and 16-level
    # chunks (64-, 32- and 16-row units: two band slabs for the first, one for the others)
    g = wl.rng(807)
    probs = [
        wl.Problem(g.integers(0, 64, size=(1, 1100, 2100)).astype(np.uint8), 64, wl.se_flat_disk(15), "dilate", "4"),
        wl.Problem(g.integers(0, 32, size=(2, 200, 330)).astype(np.uint8), 32, wl.se_full_random(g, 9, 5), "erode",
                   "8"),
        wl.Problem(g.integers(0, 256, size=(1, 150, 260)).astype(np.uint8), 256, wl.se_random(g, 11, 7, 0.5, 20),
                   "dilate", "16"),
    ]
    chunks = [ctx.plan(torch.from_numpy(p.f).cuda(), p.L, p.se, op=0 if p.op == "dilate" else 1,
                       method="direct_fp8").level_chunks for p in probs]
    assert chunks == [16, 4, 16]
    items, outs = [], []
    for p in probs:
        ft = torch.from_numpy(p.f).cuda()
        o = torch.full(ft.shape, -9, dtype=torch.int32, device="cuda")
        c = torch.full(ft.shape, -9, dtype=torch.int32, device="cuda")
        items.append((ft, p.L, p.se, p.op, o, c))
        outs.append((o, c))
    ctx.run_batch(items, method="direct_fp8")
    ctx.check()
    for p, (o, c) in zip(probs, outs):
        fn = oracle.dilate if p.op == "dilate" else oracle.erode
        rD, rC = fn(p.f, p.L, p.se.mask, p.se.offset, p.se.origin, nthreads=0)
        assert np.array_equal(o.cpu().numpy(), rD), p.name
        assert np.array_equal(c.cpu().numpy(), rC), p.name
