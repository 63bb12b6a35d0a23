"""The paper's exactness experiment (Sec. 4.3) on the GPU: 100 random 99 x 99
image / filter pairs for each odd filter size 3^2 .. 17^2, and 100 random
pairs with a 5 x 5 filter for each image size 100^2 .. 600^2, values drawn
uniformly from 0..255 for image and filter; every output must equal the
oracle's (mean absolute error exactly 0, as the paper reports).  Each group
runs as one heterogeneous AUTO batch."""
import numpy as np
import pytest

import oracle
from paper_2305_03018_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
L = 256


def _run_group(ctx, pairs):
    items, outs = [], []
    for f, se in pairs:
        ft = torch.from_numpy(f).cuda()
        o = torch.empty(f.shape, dtype=torch.int32, device="cuda")
        c = torch.empty(f.shape, dtype=torch.int32, device="cuda")
        items.append((ft, L, se, "dilate", o, c))
        outs.append((o, c))
    ctx.run_batch(items, method="auto")
    ctx.check()
    mae = 0.0
    for (f, se), (o, c) in zip(pairs, outs):
        D, cD = oracle.dilate(f, L, se.mask, se.offset, se.origin, nthreads=0)
        got = o.cpu().numpy()
        mae = max(mae, float(np.abs(got.astype(np.int64) - D).mean()))
        assert np.array_equal(c.cpu().numpy(), cD)
    return mae


@pytest.mark.parametrize("k", [3, 5, 7, 9, 11, 13, 15, 17])
def test_filter_size_series(k):
    from paper_2305_03018_gb300.morph import get_context
    g = wl.rng(4300 + k)
    pairs = [(g.integers(0, L, size=(1, 99, 99)).astype(np.uint8), wl.se_full_random(g, k, L - 1))
             for _ in range(100)]
    assert _run_group(get_context(0), pairs) == 0.0


@pytest.mark.parametrize("n", [100, 200, 300, 400, 500, 600])
def test_image_size_series(n):
    from paper_2305_03018_gb300.morph import get_context
    g = wl.rng(4400 + n)
    pairs = [(g.integers(0, L, size=(1, n, n)).astype(np.uint8), wl.se_full_random(g, 5, L - 1))
             for _ in range(100)]
    assert _run_group(get_context(0), pairs) == 0.0
