"""Pins of the composite-operator oracle (no GPU).

oracle.opening / closing / gradient apply the definitions of Sec. 2.1 twice on
the raw integers (the erosion's result may be negative; no tonal shift).  They
are pinned by
* their two one-step helpers agreeing with the plain-C oracle on images in
  [0, L) (itself pinned to the paper's examples and to brute force);
* SciPy's grey_opening / grey_closing / morphological_gradient for flat boxes
  with a centred origin on interior pixels (SciPy pads the border, these
  conventions skip it);
* the adjunction properties: opening anti-extensive and idempotent, closing
  extensive and idempotent, gradient non-negative and zero on constant images;
* hand-worked 1-D cases, including the empty-tap convention (the lowest value
  of the second pass's input range for a dilation, the highest for an
  erosion).
"""
import numpy as np
import pytest

import oracle
from paper_2305_03018_gb300 import workloads as wl


def _op(f, L, se, which):
    return {"open": oracle.opening, "close": oracle.closing, "gradient": oracle.gradient}[which](
        f, L, se.mask, se.offset, se.origin)


def test_one_step_helpers_agree_with_the_c_oracle():
    g = wl.rng(30)
    for _ in range(60):
        L = int(g.integers(2, 60))
        f = g.integers(0, L, size=(int(g.integers(1, 3)), int(g.integers(1, 20)), int(g.integers(1, 20))))
        se = wl.se_random(g, int(g.integers(1, 8)), int(g.integers(1, 8)), 0.6, int(g.integers(0, 9)),
                          origin=(int(g.integers(-2, 9)), int(g.integers(-2, 9))), force_origin=False)
        D, _ = oracle.dilate(f, L, se.mask, se.offset, se.origin)
        E, _ = oracle.erode(f, L, se.mask, se.offset, se.origin)
        assert np.array_equal(oracle._dilate_raw(f, 0, se.mask, se.offset, se.origin), D)
        assert np.array_equal(oracle._erode_raw(f, L - 1, se.mask, se.offset, se.origin), E)


@pytest.mark.parametrize("k", [3, 5, 9])
def test_flat_boxes_match_scipy_on_interior_pixels(k):
    nd = pytest.importorskip("scipy.ndimage")
    g = wl.rng(40 + k)
    f = g.integers(0, 50, size=(1, 60, 70))
    se = wl.se_flat_square(k)
    m = k - 1                                  # two passes of reach k // 2
    inner = (slice(None), slice(m, -m), slice(m, -m))
    assert np.array_equal(_op(f, 50, se, "open")[inner], nd.grey_opening(f[0], size=(k, k))[None][inner])
    assert np.array_equal(_op(f, 50, se, "close")[inner], nd.grey_closing(f[0], size=(k, k))[None][inner])
    r = k // 2
    inner1 = (slice(None), slice(r, -r), slice(r, -r))
    assert np.array_equal(_op(f, 50, se, "gradient")[inner1],
                          nd.morphological_gradient(f[0], size=(k, k))[None][inner1])


def test_adjunction_properties():
    g = wl.rng(31)
    for _ in range(120):
        L = int(g.integers(2, 40))
        H, W = int(g.integers(1, 18)), int(g.integers(1, 18))
        f = g.integers(0, L, size=(1, H, W)).astype(np.int64)
        se = wl.se_random(g, int(g.integers(1, 7)), int(g.integers(1, 7)), 0.6, int(g.integers(0, 5)))
        mb = se.max_offset
        o, c = _op(f, L, se, "open"), _op(f, L, se, "close")
        assert (o <= f).all() and (c >= f).all()
        # idempotence: the second opening's input o lies in [-max b, L - 1]; shift it into the
        # integer range the definitions take (translation commutes with both operators)
        assert np.array_equal(_op(o + mb, L + mb, se, "open") - mb, o)
        assert np.array_equal(_op(c, L + mb, se, "close"), c)
        assert (_op(f, L, se, "gradient") >= 0).all()


def test_constant_image_and_hand_worked_1d_cases():
    f = np.full((1, 9, 11), 5, np.int64)
    se = wl.se_flat_square(3)
    assert (_op(f, 8, se, "gradient") == 0).all()
    assert (_op(f, 8, se, "open") == 5).all() and (_op(f, 8, se, "close") == 5).all()
    # 1 x 4 image [0, 3, 1, 2], SE taps {0: b=1, +1: b=0} (origin at box column 0)
    f = np.array([[[0, 3, 1, 2]]])
    se = wl.SE(np.array([[1, 1]], np.uint8), np.array([[1, 0]], np.int32), (0, 0))
    # erosion E(x) = min(f(x) - 1, f(x + 1) - 0) = [min(-1, 3), min(2, 1), min(0, 2), 2 - 1]
    # (the last pixel has only tap 0) = [-1, 1, 0, 1]
    E = oracle._erode_raw(f, 3, se.mask, se.offset, se.origin)
    assert E.tolist() == [[[-1, 1, 0, 1]]]
    # opening O(x) = max(E(x) + 1, E(x - 1) + 0) = [0, max(2, -1), max(1, 1), max(2, 0)] = [0, 2, 1, 2]
    assert oracle.opening(f, 4, se.mask, se.offset, se.origin).tolist() == [[[0, 2, 1, 2]]]
    # empty-tap convention: a single tap displaced out of the 1 x 1 image
    se1 = wl.SE(np.array([[1]], np.uint8), np.array([[2]], np.int32), (0, 1))
    f1 = np.array([[[1]]])
    assert oracle.opening(f1, 4, se1.mask, se1.offset, se1.origin).tolist() == [[[-2]]]   # -max b
    assert oracle.closing(f1, 4, se1.mask, se1.offset, se1.origin).tolist() == [[[5]]]    # L - 1 + max b
