"""Pins for the oracle's dilation backward (no GPU).

* Closed form for a single-point SE: the dilation is a translation, so the
  input gradient is the translated upstream gradient and the SE gradient is
  the sum of g over the pixels that have a valid source.
* Exact central finite differences of the real-valued max-plus dilation at
  tie-free pixels.  Inputs are integers, so a unique maximum beats every other
  candidate by at least 1 and a perturbation of +-0.25 cannot change the
  argmax: the central difference is then exact.  Tied pixels get g = 0.
"""
import numpy as np

import oracle
from paper_2305_03018_gb300 import workloads as wl


def _real_dilate(f, mask, off, origin):
    """Real-valued max-plus dilation over the valid taps (cropped to F)."""
    N, H, W = f.shape
    kh, kw = mask.shape
    oy, ox = origin
    out = np.full((N, H, W), -np.inf)
    for r in range(kh):
        for c in range(kw):
            if not mask[r, c]:
                continue
            dy, dx = r - oy, c - ox
            src = np.full((N, H, W), -np.inf)
            i0, i1 = max(0, dy), min(H, H + dy)
            j0, j1 = max(0, dx), min(W, W + dx)
            if i0 < i1 and j0 < j1:
                src[:, i0:i1, j0:j1] = f[:, i0 - dy:i1 - dy, j0 - dx:j1 - dx] + off[r, c]
            out = np.maximum(out, src)
    return np.where(np.isfinite(out), out, 0.0)


def test_single_point_se_closed_form():
    g = wl.rng(21)
    f = g.integers(0, 8, size=(2, 9, 12)).astype(np.int32)
    m = np.zeros((3, 4), np.uint8)
    m[2, 0] = 1
    o = np.zeros((3, 4), np.int32)
    o[2, 0] = 3
    origin = (1, 2)                      # tap offset y = (1, -2)
    D, cD = oracle.dilate(f, 8, m, o, origin)
    up = g.standard_normal(f.shape)
    gf, gb = oracle.dilate_backward(f, 8, m, o, origin, D, cD, up)
    exp = np.zeros_like(up)
    # p receives g(p + y) when p + y is inside the image
    exp[:, 0:8, 2:12] = up[:, 1:9, 0:10]
    np.testing.assert_allclose(gf, exp, rtol=0, atol=1e-12)
    # b receives g(x) over every x whose source x - y lies inside
    assert abs(gb[2, 0] - up[:, 1:9, 0:10].sum()) < 1e-9
    assert np.count_nonzero(gb) == 1


def test_finite_differences_tie_free():
    g = wl.rng(22)
    L = 32
    f = g.integers(0, L, size=(2, 14, 15)).astype(np.int32)
    se = wl.se_full_random(g, 5, 7)
    D, cD = oracle.dilate(f, L, se.mask, se.offset, se.origin)
    up = g.standard_normal(f.shape)
    up[cD > 1] = 0.0                     # tie-split pixels excluded from the FD comparison
    gf, gb = oracle.dilate_backward(f, L, se.mask, se.offset, se.origin, D, cD, up)
    eps = 0.25
    ff = f.astype(np.float64)
    off = se.offset.astype(np.float64)

    def loss(fv, ov):
        return float((up * _real_dilate(fv, se.mask, ov, se.origin)).sum())

    for (n, i, j) in [(0, 0, 0), (0, 7, 7), (1, 13, 14), (1, 3, 10), (0, 12, 1)]:
        fp, fm = ff.copy(), ff.copy()
        fp[n, i, j] += eps
        fm[n, i, j] -= eps
        fd = (loss(fp, off) - loss(fm, off)) / (2 * eps)
        assert abs(fd - gf[n, i, j]) < 1e-9, (n, i, j, fd, gf[n, i, j])
    for (r, c) in [(0, 0), (2, 2), (4, 1), (1, 4)]:
        op, om = off.copy(), off.copy()
        op[r, c] += eps
        om[r, c] -= eps
        fd = (loss(ff, op) - loss(ff, om)) / (2 * eps)
        assert abs(fd - gb[r, c]) < 1e-9, (r, c, fd, gb[r, c])


def test_tie_split_sums_to_upstream():
    # every pixel with at least one valid tap passes exactly g(x) downstream
    g = wl.rng(23)
    f = g.integers(0, 4, size=(1, 11, 11)).astype(np.int32)   # many ties
    se = wl.se_random(g, 3, 3, 0.8, 1)
    D, cD = oracle.dilate(f, 4, se.mask, se.offset, se.origin)
    up = g.standard_normal(f.shape)
    gf, gb = oracle.dilate_backward(f, 4, se.mask, se.offset, se.origin, D, cD, up)
    total = up[cD > 0].sum()
    assert abs(gf.sum() - total) < 1e-9
    assert abs(gb.sum() - total) < 1e-9


def _real_erode(f, mask, off, origin):
    """Real-valued min-plus erosion over the valid taps (cropped to F)."""
    N, H, W = f.shape
    kh, kw = mask.shape
    oy, ox = origin
    out = np.full((N, H, W), np.inf)
    for r in range(kh):
        for c in range(kw):
            if not mask[r, c]:
                continue
            dy, dx = r - oy, c - ox                       # source x + y
            src = np.full((N, H, W), np.inf)
            i0, i1 = max(0, -dy), min(H, H - dy)
            j0, j1 = max(0, -dx), min(W, W - dx)
            if i0 < i1 and j0 < j1:
                src[:, i0:i1, j0:j1] = f[:, i0 + dy:i1 + dy, j0 + dx:j1 + dx] - off[r, c]
            out = np.minimum(out, src)
    return np.where(np.isfinite(out), out, 0.0)


def test_erosion_finite_differences_tie_free():
    g = wl.rng(24)
    L = 32
    f = g.integers(0, L, size=(2, 13, 16)).astype(np.int32)
    se = wl.se_random(g, 5, 3, 0.8, 7, origin=(1, 2))
    E, cE = oracle.erode(f, L, se.mask, se.offset, se.origin)
    up = g.standard_normal(f.shape)
    up[cE != 1] = 0.0                      # ties and empty pixels excluded
    gf, gb = oracle.erode_backward(f, L, se.mask, se.offset, se.origin, E, cE, up)
    eps = 0.25
    ff, off = f.astype(np.float64), se.offset.astype(np.float64)

    def loss(fv, ov):
        return float((up * _real_erode(fv, se.mask, ov, se.origin)).sum())

    for (n, i, j) in [(0, 0, 0), (1, 6, 8), (0, 12, 15), (1, 2, 1)]:
        fp, fm = ff.copy(), ff.copy()
        fp[n, i, j] += eps
        fm[n, i, j] -= eps
        assert abs((loss(fp, off) - loss(fm, off)) / (2 * eps) - gf[n, i, j]) < 1e-9
    for (r, c) in zip(*np.nonzero(se.mask)):
        op, om = off.copy(), off.copy()
        op[r, c] += eps
        om[r, c] -= eps
        assert abs((loss(ff, op) - loss(ff, om)) / (2 * eps) - gb[r, c]) < 1e-9


def test_erosion_single_point_closed_form():
    g = wl.rng(25)
    f = g.integers(0, 8, size=(1, 9, 10)).astype(np.int32)
    m = np.zeros((3, 3), np.uint8)
    m[2, 0] = 1                            # y = (1, -1): E(x) = f(x + y) - b
    o = np.zeros((3, 3), np.int32)
    o[2, 0] = 2
    E, cE = oracle.erode(f, 8, m, o, (1, 1))
    up = g.standard_normal(f.shape)
    gf, gb = oracle.erode_backward(f, 8, m, o, (1, 1), E, cE, up)
    exp = np.zeros_like(up)
    exp[:, 1:9, 0:9] = up[:, 0:8, 1:10]    # p = x + y receives g(x)
    np.testing.assert_allclose(gf, exp, rtol=0, atol=1e-12)
    assert abs(gb[2, 0] + up[:, 0:8, 1:10].sum()) < 1e-9
