"""Pins for the 3-D oracle (no GPU): a 1-slice SE reduces to the 2-D
oracle slice by slice (itself pinned), a single-point 3-D SE is a 3-D
translation, 3-D duality holds, and tiny volumes match an independent
brute force over all (source, tap) pairs."""
import itertools

import numpy as np

import oracle
from paper_2305_03018_gb300 import workloads as wl


def test_one_slice_se_equals_2d_per_slice():
    g = wl.rng(41)
    f = g.integers(0, 16, size=(2, 5, 11, 9)).astype(np.int32)
    se = wl.se_random(g, 5, 3, 0.6, 3, origin=(1, 2))
    D3, C3 = oracle.dilate3d(f, 16, se.mask[None], se.offset[None], (0,) + se.origin)
    E3, F3 = oracle.erode3d(f, 16, se.mask[None], se.offset[None], (0,) + se.origin)
    D2, C2 = oracle.dilate(f.reshape(-1, 11, 9), 16, se.mask, se.offset, se.origin)
    E2, F2 = oracle.erode(f.reshape(-1, 11, 9), 16, se.mask, se.offset, se.origin)
    assert (D3.reshape(-1, 11, 9) == D2).all() and (C3.reshape(-1, 11, 9) == C2).all()
    assert (E3.reshape(-1, 11, 9) == E2).all() and (F3.reshape(-1, 11, 9) == F2).all()


def test_single_point_is_translation_3d():
    g = wl.rng(42)
    f = g.integers(0, 8, size=(1, 6, 7, 8)).astype(np.int32)
    m = np.zeros((3, 2, 3), np.uint8)
    m[2, 0, 1] = 1
    o = np.zeros((3, 2, 3), np.int32)
    o[2, 0, 1] = 4
    D, C = oracle.dilate3d(f, 8, m, o, (1, 1, 1))      # y = (1, -1, 0)
    exp = np.zeros_like(f)
    exp[:, 1:, :6, :] = f[:, :5, 1:, :] + 4
    assert (D == exp).all()
    valid = np.zeros_like(f)
    valid[:, 1:, :6, :] = 1                            # x - y inside the volume
    assert (C == valid).all()


def test_duality_3d():
    g = wl.rng(43)
    L = 20
    f = g.integers(0, L, size=(1, 6, 8, 7)).astype(np.int32)
    m = (g.random((3, 3, 4)) < 0.5).astype(np.uint8)
    m[1, 1, 1] = 1
    o = (g.integers(0, 5, size=m.shape) * m).astype(np.int32)
    E, cE = oracle.erode3d(f, L, m, o, (1, 1, 1))
    D, cD = oracle.dilate3d((L - 1) - f, L, m[::-1, ::-1, ::-1].copy(), o[::-1, ::-1, ::-1].copy(), (1, 1, 2))
    assert (E == (L - 1) - D).all() and (cE == cD).all()


def test_tiny_brute_force():
    g = wl.rng(44)
    for _ in range(40):
        Z, H, W = (int(g.integers(1, 4)) for _ in range(3))
        L = int(g.integers(2, 6))
        f = g.integers(0, L, size=(1, Z, H, W)).astype(np.int32)
        kd, kh, kw = (int(g.integers(1, 3)) for _ in range(3))
        m = (g.random((kd, kh, kw)) < 0.7).astype(np.uint8)
        o = (g.integers(0, 3, size=m.shape) * m).astype(np.int32)
        org = tuple(int(g.integers(0, k)) for k in (kd, kh, kw))
        D, cD = oracle.dilate3d(f, L, m, o, org)
        ref = np.zeros_like(f)
        cnt = np.zeros_like(f)
        best = {}
        for (z, i, j) in itertools.product(range(Z), range(H), range(W)):       # every source pixel
            for (q, r, c) in zip(*np.nonzero(m)):                               # every tap
                x = (z + q - org[0], i + r - org[1], j + c - org[2])
                if all(0 <= x[a] < (Z, H, W)[a] for a in range(3)):
                    best.setdefault(x, []).append(f[0, z, i, j] + o[q, r, c])
        for x, vals in best.items():
            ref[(0,) + x] = max(vals)
            cnt[(0,) + x] = vals.count(max(vals))
        assert (D == ref).all() and (cD == cnt).all()
