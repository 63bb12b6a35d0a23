"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself:

* the values the paper prints for its worked example (Examples 2-5);
* an independent set-algebra brute force on tiny inputs: the umbra of the
  dilation is the Minkowski sum of the umbras, and the umbra of the erosion
  is their Minkowski difference (the classical umbra homomorphism the
  paper's Step 1 construction is named after);
* a library routine the special case reduces to (SciPy's grey dilation and
  erosion for odd full-box SEs with a centred origin);
* closed forms (pure translation, constant image, identity) and invariants
  (duality, monotonicity, composition, count-polynomial mass).
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_2305_03018_gb300 import workloads as wl
from tests.conftest import GOLDEN


def _example():
    with open(os.path.join(GOLDEN, "example2_5.json")) as fh:
        ex = json.load(fh)
    f = np.array(ex["image"], np.int32)[None, None, :]
    flt = ex["filter"]
    mask = np.array([[0 if v is None else 1 for v in flt]], np.uint8)
    off = np.array([[0 if v is None else v for v in flt]], np.int32)
    origin = (0, ex["filter_origin"])
    assert ex["image_origin"] == 0
    return ex, f, mask, off, origin


# ------------------------------------------------------------ paper example
def test_example2_dilation_values():
    ex, f, mask, off, origin = _example()
    D, cD = oracle.dilate(f, ex["L"], mask, off, origin)
    assert D.ravel().tolist() == ex["dilation"]


def test_example5_count_polynomial():
    ex, f, mask, off, origin = _example()
    D, cD, C = oracle.dilate(f, ex["L"], mask, off, origin, counts=True)
    printed = np.array(ex["count_umbra_printed"])       # row 0 = top grey level
    R = printed.shape[0]
    assert C.shape[-1] == R                              # l_R + 1 = 7 + 2 + 1 degrees
    got = C[0, 0].T[::-1]                                # [degree top..0][x]
    np.testing.assert_array_equal(got, printed)
    col2 = np.array(ex["count_column_x2_example4"])
    np.testing.assert_array_equal(C[0, 0, 2][::-1], col2)
    # Eq. 9: the dilation is the top nonzero degree; its coefficient is cD
    for x in range(6):
        top = max(d for d in range(R) if C[0, 0, x, d] >= 1)
        assert top == D[0, 0, x]
        assert C[0, 0, x, top] == cD[0, 0, x]


def test_example3_umbras_are_one_hot_of_values():
    # Eq. 7/8 read back from the printed umbras: column x has its single 1 at
    # row (from the bottom) f(x), resp. b(y); columns outside B are all zero.
    ex, f, mask, off, origin = _example()
    fu = np.array(ex["f_umbra_printed"])[::-1]
    bu = np.array(ex["b_umbra_printed"])[::-1]
    assert [int(np.argmax(fu[:, x])) for x in range(6)] == ex["image"]
    assert fu.sum(axis=0).tolist() == [1] * 6
    for y, v in enumerate(ex["filter"]):
        if v is None:
            assert bu[:, y].sum() == 0
        else:
            assert bu[:, y].sum() == 1 and int(np.argmax(bu[:, y])) == v


# ------------------------------------------------ umbra set-algebra brute force
def _umbra_dilate(f, L, mask, off, origin):
    """Top surface of the Minkowski sum of the two (truncated) umbras."""
    H, W = f.shape
    oy, ox = origin
    pts = {}
    for i, j in itertools.product(range(H), range(W)):
        for r, c in itertools.product(range(mask.shape[0]), range(mask.shape[1])):
            if not mask[r, c]:
                continue
            for v in range(0, f[i, j] + 1):
                for w in range(0, off[r, c] + 1):
                    x = (i + r - oy, j + c - ox)
                    pts[x] = max(pts.get(x, -1), v + w)
    out = np.zeros((H, W), np.int64)
    for i, j in itertools.product(range(H), range(W)):
        out[i, j] = pts.get((i, j), 0)
    return out


def _umbra_erode(f, L, mask, off, origin):
    """Largest h such that the SE umbra translated to (x, h) fits in the image umbra."""
    H, W = f.shape
    oy, ox = origin
    maxb = max([int(off[r, c]) for r, c in zip(*np.nonzero(mask))] or [0])
    out = np.zeros((H, W), np.int64)
    for i, j in itertools.product(range(H), range(W)):
        best = None
        for h in range(L - 1, -maxb - 2, -1):
            ok = True
            for r, c in zip(*np.nonzero(mask)):
                si, sj = i + r - oy, j + c - ox
                if 0 <= si < H and 0 <= sj < W:
                    # every umbra point (y, w <= b(y)) lifted by h must lie under f
                    if h + off[r, c] > f[si, sj]:
                        ok = False
                        break
            if ok:
                best = h
                break
        out[i, j] = best
    return out


def _tiny_cases():
    g = wl.rng(12345)
    cases = []
    # all 1x3 images over L=3 with every 1x2 / 1x3 SE (offsets <= 1) and every origin
    for fv in itertools.product(range(3), repeat=3):
        f = np.array([fv], np.int32)
        for kw in (2, 3):
            for mbits in itertools.product((0, 1), repeat=kw):
                if not any(mbits):
                    continue
                for obits in itertools.product((0, 1), repeat=kw):
                    for ox in range(kw):
                        m = np.array([mbits], np.uint8)
                        o = np.array([obits], np.int32) * m
                        cases.append((f, 3, m, o.astype(np.int32), (0, ox)))
    # random 2-D tiny cases, including origins outside the support and empty B
    for _ in range(300):
        H, W = int(g.integers(1, 4)), int(g.integers(1, 4))
        L = int(g.integers(2, 5))
        kh, kw = int(g.integers(1, 4)), int(g.integers(1, 4))
        f = g.integers(0, L, size=(H, W)).astype(np.int32)
        m = (g.random((kh, kw)) < 0.6).astype(np.uint8)
        o = (g.integers(0, 3, size=(kh, kw)) * m).astype(np.int32)
        origin = (int(g.integers(0, kh)), int(g.integers(0, kw)))
        cases.append((f, L, m, o, origin))
    return cases


def test_exhaustive_tiny_dilation_matches_umbra_minkowski_sum():
    for f, L, m, o, origin in _tiny_cases():
        D, _ = oracle.dilate(f, L, m, o, origin)
        np.testing.assert_array_equal(D[0], _umbra_dilate(f, L, m, o, origin),
                                      err_msg=f"f={f.tolist()} m={m.tolist()} o={o.tolist()} org={origin}")


def test_exhaustive_tiny_erosion_matches_umbra_minkowski_difference():
    for f, L, m, o, origin in _tiny_cases():
        E, _ = oracle.erode(f, L, m, o, origin)
        np.testing.assert_array_equal(E[0], _umbra_erode(f, L, m, o, origin),
                                      err_msg=f"f={f.tolist()} m={m.tolist()} o={o.tolist()} org={origin}")


def test_paper_exactness_protocol_small():
    # Sec. 4.3 protocol (random 0..255 images and filters), scaled down: the
    # count polynomial's top degree (Step 3) must equal the sliding max.
    g = wl.rng(7)
    for k in (3, 5, 7):
        f = g.integers(0, 256, size=(1, 23, 23)).astype(np.int32)
        se = wl.se_full_random(g, k, 255)
        D, cD, C = oracle.dilate(f, 256, se.mask, se.offset, se.origin, counts=True)
        R = C.shape[-1]
        top = np.where(C.sum(-1) > 0, R - 1 - np.argmax(C[..., ::-1] > 0, axis=-1), 0)
        np.testing.assert_array_equal(top, D)


# ---------------------------------------------------------- library special case
def test_scipy_grey_dilation_and_erosion_full_box():
    ndi = pytest.importorskip("scipy.ndimage")
    g = wl.rng(99)
    for (H, W, k, L, mo) in [(17, 23, 3, 16, 3), (31, 19, 5, 64, 7), (12, 40, 7, 256, 15), (9, 9, 9, 8, 0)]:
        f = g.integers(0, L, size=(H, W)).astype(np.int64)
        off = g.integers(0, mo + 1, size=(k, k)).astype(np.int64)
        m = np.ones((k, k), np.uint8)
        ref_d = ndi.grey_dilation(f, structure=off, mode="constant", cval=-(10 ** 9))
        ref_e = ndi.grey_erosion(f, structure=off, mode="constant", cval=10 ** 9)
        D, _ = oracle.dilate(f, L, m, off, (k // 2, k // 2))
        E, _ = oracle.erode(f, L, m, off, (k // 2, k // 2))
        np.testing.assert_array_equal(D[0], ref_d)
        np.testing.assert_array_equal(E[0], ref_e)


# ------------------------------------------------------------ closed forms
def test_single_point_se_is_translation():
    g = wl.rng(3)
    f = g.integers(0, 16, size=(1, 13, 11)).astype(np.int32)
    for (kh, kw, r, c, oy, ox, val) in [(3, 3, 0, 2, 1, 1, 5), (5, 4, 4, 0, 0, 3, 0), (1, 1, 0, 0, 0, 0, 2)]:
        m = np.zeros((kh, kw), np.uint8)
        m[r, c] = 1
        o = np.zeros((kh, kw), np.int32)
        o[r, c] = val
        D, cD = oracle.dilate(f, 16, m, o, (oy, ox))
        dy, dx = r - oy, c - ox
        exp = np.zeros_like(f)
        expc = np.zeros_like(f)
        for i in range(13):
            for j in range(11):
                si, sj = i - dy, j - dx
                if 0 <= si < 13 and 0 <= sj < 11:
                    exp[0, i, j] = f[0, si, sj] + val
                    expc[0, i, j] = 1
        np.testing.assert_array_equal(D, exp)
        np.testing.assert_array_equal(cD, expc)


def test_constant_image_flat_box_counts_valid_taps():
    sig = pytest.importorskip("scipy.signal")
    for (H, W, k, a) in [(20, 30, 5, 7), (8, 8, 9, 0), (63, 70, 63, 3)]:
        f = np.full((1, H, W), a, np.int32)
        se = wl.se_flat_square(k)
        D, cD = oracle.dilate(f, 8, se.mask, se.offset, se.origin)
        assert (D == a).all()
        valid = sig.correlate2d(np.ones((H, W)), np.ones((k, k)), mode="same")
        np.testing.assert_array_equal(cD[0], valid.round().astype(np.int32))
    # the largest count the library must represent: a 63x63 flat SE, interior pixel
    f = np.full((1, 63, 63), 5, np.int32)
    se = wl.se_flat_square(63)
    _, cD = oracle.dilate(f, 8, se.mask, se.offset, se.origin)
    assert cD[0, 31, 31] == 63 * 63


def test_flat_1x1_is_identity():
    g = wl.rng(4)
    f = g.integers(0, 256, size=(2, 9, 14)).astype(np.int32)
    se = wl.se_flat_square(1)
    D, cD = oracle.dilate(f, 256, se.mask, se.offset, se.origin)
    E, cE = oracle.erode(f, 256, se.mask, se.offset, se.origin)
    np.testing.assert_array_equal(D, f)
    np.testing.assert_array_equal(E, f)
    assert (cD == 1).all() and (cE == 1).all()


def test_empty_support_conventions():
    f = np.arange(12, dtype=np.int32).reshape(1, 3, 4)
    m = np.zeros((3, 3), np.uint8)
    o = np.zeros((3, 3), np.int32)
    D, cD = oracle.dilate(f, 16, m, o, (1, 1))
    E, cE = oracle.erode(f, 16, m, o, (1, 1))
    assert (D == 0).all() and (cD == 0).all()           # Eq. 6: x not in F (+) B
    assert (E == 15).all() and (cE == 0).all()          # duality reading: l = L - 1


# ------------------------------------------------------------- invariants
def _reflect(mask, off, origin):
    kh, kw = mask.shape
    return mask[::-1, ::-1].copy(), off[::-1, ::-1].copy(), (kh - 1 - origin[0], kw - 1 - origin[1])


def test_duality_erosion_vs_dilation_of_negative():
    g = wl.rng(5)
    for L, k, mo, org in [(16, 5, 3, None), (64, 7, 7, (0, 6)), (256, 3, 15, (2, 0))]:
        f = g.integers(0, L, size=(2, 21, 17)).astype(np.int32)
        se = wl.se_random(g, k, k, 0.5, mo, origin=org)
        E, cE = oracle.erode(f, L, se.mask, se.offset, se.origin)
        m2, o2, org2 = _reflect(se.mask, se.offset, se.origin)
        D, cD = oracle.dilate((L - 1) - f, L, m2, o2, org2)
        np.testing.assert_array_equal(E, (L - 1) - D)
        np.testing.assert_array_equal(cE, cD)


def test_monotone_in_image_and_offsets():
    g = wl.rng(6)
    f = g.integers(0, 32, size=(1, 25, 25)).astype(np.int32)
    f2 = np.minimum(f + g.integers(0, 3, size=f.shape).astype(np.int32), 31)
    se = wl.se_random(g, 5, 5, 0.7, 4)
    o2 = se.offset + g.integers(0, 2, size=se.offset.shape).astype(np.int32) * se.mask
    D1, _ = oracle.dilate(f, 32, se.mask, se.offset, se.origin)
    D2, _ = oracle.dilate(f2, 32, se.mask, se.offset, se.origin)
    D3, _ = oracle.dilate(f, 32, se.mask, o2, se.origin)
    assert (D2 >= D1).all() and (D3 >= D1).all()


def test_count_mass_equals_valid_taps():
    sig = pytest.importorskip("scipy.signal")
    g = wl.rng(8)
    f = g.integers(0, 16, size=(1, 19, 27)).astype(np.int32)
    se = wl.se_random(g, 7, 5, 0.5, 3, origin=(1, 4))
    _, _, C = oracle.dilate(f, 16, se.mask, se.offset, se.origin, counts=True)
    # valid taps at x = #{y in B : x - y in F}: a convolution of F's indicator with the mask
    kh, kw = se.mask.shape
    oy, ox = se.origin
    full = sig.convolve2d(np.ones((19, 27)), se.mask.astype(float), mode="full")
    valid = full[oy:oy + 19, ox:ox + 27].round().astype(np.int64)
    np.testing.assert_array_equal(C.sum(-1)[0], valid)
    # first moment: sum_d d C[x, d] = sum over valid taps of f(x - y) + b(y)
    ff = sig.convolve2d(f[0].astype(float), se.mask.astype(float), mode="full")[oy:oy + 19, ox:ox + 27]
    bb = sig.convolve2d(np.ones((19, 27)), (se.offset * se.mask).astype(float), mode="full")[oy:oy + 19, ox:ox + 27]
    mom = (C[0] * np.arange(C.shape[-1])).sum(-1)
    np.testing.assert_array_equal(mom, (ff + bb).round().astype(np.int64))


def _compose(s1, s2):
    """Max-plus composition b1 (+) b2 on B1 (+) B2 (origins add)."""
    k1h, k1w = s1.mask.shape
    k2h, k2w = s2.mask.shape
    kh, kw = k1h + k2h - 1, k1w + k2w - 1
    m = np.zeros((kh, kw), np.uint8)
    o = np.full((kh, kw), -1, np.int64)
    for (r1, c1) in zip(*np.nonzero(s1.mask)):
        for (r2, c2) in zip(*np.nonzero(s2.mask)):
            r, c = r1 + r2, c1 + c2
            m[r, c] = 1
            o[r, c] = max(o[r, c], s1.offset[r1, c1] + s2.offset[r2, c2])
    o[m == 0] = 0
    origin = (s1.origin[0] + s2.origin[0], s1.origin[1] + s2.origin[1])
    return m, o.astype(np.int32), origin


def test_composition_on_interior():
    g = wl.rng(9)
    L = 16
    f = g.integers(0, L, size=(1, 30, 30)).astype(np.int32)
    s1 = wl.se_random(g, 3, 5, 0.6, 2)
    s2 = wl.se_random(g, 5, 3, 0.6, 3)
    D1, _ = oracle.dilate(f, L, s1.mask, s1.offset, s1.origin)
    L2 = L + s1.max_offset
    D12, _ = oracle.dilate(D1, L2, s2.mask, s2.offset, s2.origin)
    m, o, org = _compose(s1, s2)
    Dc, _ = oracle.dilate(f, L, m, o, org)
    reach = max(s2.mask.shape)
    sl = (0, slice(reach, 30 - reach), slice(reach, 30 - reach))
    np.testing.assert_array_equal(D12[sl], Dc[sl])


def test_rows_sample_matches_full():
    g = wl.rng(10)
    f = g.integers(0, 64, size=(1, 40, 33)).astype(np.int32)
    se = wl.se_random(g, 9, 9, 0.5, 7)
    D, cD = oracle.dilate(f, 64, se.mask, se.offset, se.origin)
    Ds, cDs = oracle.dilate(f, 64, se.mask, se.offset, se.origin, rows=(10, 17), nthreads=2)
    np.testing.assert_array_equal(Ds[:, 10:17], D[:, 10:17])
    np.testing.assert_array_equal(cDs[:, 10:17], cD[:, 10:17])


def test_rejects_out_of_range_input():
    f = np.array([[[0, 16]]], np.int32)
    with pytest.raises(ValueError):
        oracle.dilate(f, 16, np.ones((1, 1), np.uint8), np.zeros((1, 1), np.int32), (0, 0))
    with pytest.raises(ValueError):
        oracle.dilate(f * 0, 16, np.ones((1, 1), np.uint8), -np.ones((1, 1), np.int32), (0, 0))
