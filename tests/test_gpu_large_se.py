"""SEs larger than 63x63 (up to 255x255), as in the paper's runtime
experiments, on every route, against the oracle on sampled rows."""
import numpy as np
import pytest

import oracle
from paper_2305_03018_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method", ["direct_fp8", "fft_f64", "auto"])
def test_large_non_flat_se(method):
    from paper_2305_03018_gb300.morph import get_context
    ctx = get_context(0)
    g = wl.rng(808)
    f = g.integers(0, 16, size=(1, 300, 260)).astype(np.uint8)
    se = wl.se_random(g, 121, 101, 0.8, 15, origin=(30, 70))
    ft = torch.from_numpy(f).cuda()
    for op in ("dilate", "erode"):
        fn = ctx.dilate if op == "dilate" else ctx.erode
        D, cD = fn(ft, 16, se, method=method, count=True)
        ctx.check()
        D, cD = D.cpu().numpy(), cD.cpu().numpy()
        ofn = oracle.dilate if op == "dilate" else oracle.erode
        for rows in [(0, 2), (150, 152), (298, 300)]:
            rD, rC = ofn(f, 16, se.mask, se.offset, se.origin, rows=rows, nthreads=0)
            sl = (slice(None), slice(*rows))
            assert np.array_equal(D[sl], rD[sl]) and np.array_equal(cD[sl], rC[sl]), (op, rows)


def test_512_box_is_accepted_and_513_rejected():
    from paper_2305_03018_gb300.morph import MORPH_E_INVAL, MorphError, get_context
    ctx = get_context(0)
    f = torch.zeros((1, 20, 20), dtype=torch.uint8, device="cuda")
    ok = wl.se_flat_square(511)
    D = ctx.dilate(f, 4, ok)
    ctx.check()
    assert int(D.max()) == 0
    bad = wl.SE(np.ones((513, 1), np.uint8), np.zeros((513, 1), np.int32), (0, 0))
    with pytest.raises(MorphError) as ei:
        ctx.dilate(f, 4, bad)
    assert ei.value.status == MORPH_E_INVAL
