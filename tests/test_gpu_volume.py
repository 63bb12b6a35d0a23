"""GPU 3-D dilation / erosion against the 3-D oracle, bit-exact (values and
top counts), over every route, with empty SE slices, off-centre origins and a
ragged volume."""
import numpy as np
import pytest

import oracle
from paper_2305_03018_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (N, Z, H, W, L, kd, kh, kw, p_in, max_off, origin)
CASES = [
    (1, 9, 37, 45, 16, 3, 3, 3, 0.6, 3, (1, 1, 1)),
    (2, 6, 64, 70, 64, 5, 5, 7, 0.5, 9, (0, 4, 2)),
    (1, 17, 33, 130, 256, 3, 9, 9, 0.8, 20, (2, 4, 4)),
    (1, 4, 20, 20, 8, 7, 3, 3, 1.0, 0, (3, 1, 1)),           # flat box, SE deeper than the volume
]


def _case(case):
    N, Z, H, W, L, kd, kh, kw, p_in, mo, origin = case
    g = wl.rng(sum(case[:8]) * 31 + 7)
    f = g.integers(0, L, size=(N, Z, H, W)).astype(np.uint8 if L <= 256 else np.uint16)
    m = (g.random((kd, kh, kw)) < p_in).astype(np.uint8)
    m[origin] = 1
    if kd > 2:
        m[1] = 0                                               # an empty SE slice
    o = (g.integers(0, mo + 1, size=m.shape) * m).astype(np.int32)
    return f, L, m, o, origin


@pytest.mark.parametrize("method", ["auto", "direct_fp8", "fft_f64", "ntt"])
@pytest.mark.parametrize("case", CASES)
def test_volume_bit_exact(case, method):
    from paper_2305_03018_gb300.morph import get_context
    ctx = get_context(0)
    f, L, m, o, origin = _case(case)
    ft = torch.from_numpy(f).cuda()
    for op, ref in ((0, oracle.dilate3d), (1, oracle.erode3d)):
        run = ctx.dilate3d if op == 0 else ctx.erode3d
        v, c = run(ft, L, m, o, origin, method=method, count=True)
        ctx.check()
        ev, ec = ref(f.astype(np.int32), L, m, o, origin, nthreads=4)
        assert np.array_equal(v.cpu().numpy(), ev), op
        assert np.array_equal(c.cpu().numpy(), ec), op


def test_volume_fft32_within_bound():
    # FP32 route under its proven bound is exact as well
    from paper_2305_03018_gb300.morph import get_context
    ctx = get_context(0)
    f, L, m, o, origin = _case((1, 8, 48, 48, 16, 3, 5, 5, 0.7, 2, (1, 2, 2)))
    ft = torch.from_numpy(f).cuda()
    v, c = ctx.dilate3d(ft, L, m, o, origin, method="fft_f32", count=True)
    ctx.check()
    ev, ec = oracle.dilate3d(f.astype(np.int32), L, m, o, origin, nthreads=4)
    assert np.array_equal(v.cpu().numpy(), ev) and np.array_equal(c.cpu().numpy(), ec)


def test_volume_empty_se_and_one_slice():
    from paper_2305_03018_gb300.morph import get_context
    ctx = get_context(0)
    g = wl.rng(77)
    f = g.integers(0, 10, size=(1, 3, 12, 14)).astype(np.uint8)
    ft = torch.from_numpy(f).cuda()
    m = np.zeros((2, 3, 3), np.uint8)
    o = np.zeros((2, 3, 3), np.int32)
    v, c = ctx.erode3d(ft, 10, m, o, (0, 1, 1), count=True)
    ctx.check()
    assert (v.cpu().numpy() == 9).all() and (c.cpu().numpy() == 0).all()
    # a one-slice SE is the 2-D operator slice by slice
    se = wl.se_random(g, 5, 5, 0.7, 4)
    v3 = ctx.dilate3d(ft, 10, se.mask[None], se.offset[None], (0,) + se.origin)
    v2 = ctx.dilate(ft[0], 10, se)
    ctx.check()
    assert torch.equal(v3[0], v2)
