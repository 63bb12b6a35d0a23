"""GPU composite operators (opening, closing, Beucher gradient) against the
oracle's composites (the definitions applied twice on the raw integers),
bit-exact."""
import numpy as np
import pytest

import oracle
from paper_2305_03018_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    (2, 40, 57, 16, 7, 7, 0.5, 3, None),
    (1, 64, 33, 64, 9, 15, 0.6, 7, (2, 10)),
    (1, 30, 90, 200, 5, 5, 1.0, 40, None),
    (1, 50, 50, 32, 15, 15, 1.0, 0, None),            # flat box
]


@pytest.mark.parametrize("method", ["direct_fp8", "fft_f64", "ntt"])
@pytest.mark.parametrize("case", CASES)
def test_composites_bit_exact(case, method):
    from paper_2305_03018_gb300.morph import get_context
    ctx = get_context(0)
    N, H, W, L, kh, kw, p_in, mo, origin = case
    g = wl.rng(hash(case) & 0xFFFF)
    f = g.integers(0, L, size=(N, H, W)).astype(np.uint8)
    se = wl.se_random(g, kh, kw, p_in, mo, origin=origin)
    ft = torch.from_numpy(f).cuda()
    for which, ref in (("open", oracle.opening), ("close", oracle.closing), ("gradient", oracle.gradient)):
        got = ctx.composite(which, ft, L, se, method=method)
        ctx.check()
        exp = ref(f, L, se.mask, se.offset, se.origin)
        assert np.array_equal(got.cpu().numpy(), exp), which


def test_opening_refused_beyond_tonal_limit():
    from paper_2305_03018_gb300.morph import MORPH_E_UNSUPPORTED, MorphError, get_context
    ctx = get_context(0)
    f = torch.zeros((1, 8, 8), dtype=torch.uint8, device="cuda")
    se = wl.se_full_random(wl.rng(1), 3, 20)
    with pytest.raises(MorphError) as ei:
        ctx.composite("open", f, 250, se)
    assert ei.value.status == MORPH_E_UNSUPPORTED
