"""Pins for composite operators built from the oracle (no GPU): opening is
anti-extensive and idempotent, closing extensive and idempotent, and the
Beucher gradient is non-negative and zero on constant images -- properties
of the adjunction between erosion and dilation that hold with the bounded-
domain conventions of Sec. 2.1."""
import numpy as np

import oracle
from paper_2305_03018_gb300 import workloads as wl


def opening(f, L, se):
    mb = se.max_offset
    E, _ = oracle.erode(f, L, se.mask, se.offset, se.origin)
    D, _ = oracle.dilate(E + mb, L + mb, se.mask, se.offset, se.origin)
    return D - mb


def closing(f, L, se):
    mb = se.max_offset
    D, _ = oracle.dilate(f, L, se.mask, se.offset, se.origin)
    E, _ = oracle.erode(D, L + mb, se.mask, se.offset, se.origin)
    return E


def gradient(f, L, se):
    D, _ = oracle.dilate(f, L, se.mask, se.offset, se.origin)
    E, _ = oracle.erode(f, L, se.mask, se.offset, se.origin)
    return D - E


def test_adjunction_properties():
    g = wl.rng(31)
    for _ in range(120):
        L = int(g.integers(2, 40))
        H, W = int(g.integers(1, 18)), int(g.integers(1, 18))
        f = g.integers(0, L, size=(1, H, W)).astype(np.int32)
        se = wl.se_random(g, int(g.integers(1, 7)), int(g.integers(1, 7)), 0.6, int(g.integers(0, 5)))
        o, c = opening(f, L, se), closing(f, L, se)
        assert (o <= f).all() and (c >= f).all()
        if o.min() >= 0:                              # idempotence (second opening on the same range)
            assert (opening(o, L, se) == o).all()
        mb = se.max_offset
        assert (closing(c, L + mb, se) == c).all()
        assert (gradient(f, L, se) >= 0).all()


def test_gradient_of_constant_image_is_flat_se_zero():
    f = np.full((1, 9, 11), 5, np.int32)
    se = wl.se_flat_square(3)
    assert (gradient(f, 8, se) == 0).all()
