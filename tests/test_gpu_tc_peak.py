"""The tensor-pipe peak measurement hook (morph_tc_fp8_peak) on the GPU.

It issues the FP8 route's MMA shape back to back on every SM.  The rate must
be positive and physically plausible for one GB300 (between the measured
cuBLAS bf16 rate and eight times it), must not raise the device error word,
and must leave the context usable (an FP8 dilation afterwards is exact)."""
import numpy as np
import pytest

import oracle
from paper_2305_03018_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_peak_is_plausible_and_leaves_the_context_usable():
    from paper_2305_03018_gb300.morph import get_context
    ctx = get_context(0)
    tf = ctx.tc_fp8_peak()
    ctx.check()
    assert 1000.0 < tf < 16000.0, tf
    g = wl.rng(931)
    f = g.integers(0, 64, size=(1, 300, 400)).astype(np.uint8)
    se = wl.se_flat_disk(9)
    D, cD = ctx.dilate(torch.from_numpy(f).cuda(), 64, se, method="direct_fp8", count=True)
    ctx.check()
    rD, rC = oracle.dilate(f, 64, se.mask, se.offset, se.origin, nthreads=0)
    assert np.array_equal(D.cpu().numpy(), rD) and np.array_equal(cD.cpu().numpy(), rC)
