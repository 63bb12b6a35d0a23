"""The allocation-free entry point (morph_run_noalloc) against the oracle and
the regular entry point.

Some callers cannot allocate device memory; morph_run_noalloc serves them
from a fixed 64 MiB device array.  This file is collected last so that a run
stopping at its first failure has already run every other test.  It must
pass alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import oracle
from paper_2305_03018_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(f_t, L, se, op):
    from paper_2305_03018_gb300 import morph as M
    img = M.make_image(f_t, L)
    sv = M.se_view(se)
    shape = (img.n, img.h, img.w)
    out = torch.full(shape, -7, dtype=torch.int32, device=f_t.device)
    cnt = torch.full(shape, -7, dtype=torch.int32, device=f_t.device)
    status = torch.full((1,), 12345, dtype=torch.int32, device=f_t.device)
    rc = M.morph_run_noalloc(img, sv.c, op, out.data_ptr(), cnt.data_ptr(), status.data_ptr(),
                             M.current_stream_handle(f_t.device))
    return rc, out, cnt, status


def test_noalloc_matches_regular_entry_point_on_two_calls_in_a_row():
    from paper_2305_03018_gb300.morph import MORPH_OK, get_context
    ctx = get_context(0)
    g = wl.rng(4242)
    calls = [
        (g.integers(0, 64, size=(2, 45, 150)).astype(np.uint8), 64, wl.se_random(g, 9, 11, 0.6, 7, origin=(2, 8)), 0),
        (g.integers(0, 256, size=(1, 70, 101)).astype(np.uint8), 256, wl.se_random_convex(g, 15, 12, 15), 1),
    ]
    for f_np, L, se, op in calls:                # two calls in a row, sharing the scratch
        f_t = torch.from_numpy(f_np).cuda()
        rc, out, cnt, status = _noalloc(f_t, L, se, op)
        assert rc == MORPH_OK
        fn = ctx.dilate if op == 0 else ctx.erode
        ref, ref_c = fn(f_t, L, se, method="direct_fp8", count=True)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(out, ref)             # bit-exact, as every parity test here
        assert torch.equal(cnt, ref_c)
        ofn = oracle.dilate if op == 0 else oracle.erode
        oD, oC = ofn(f_np, L, se.mask, se.offset, se.origin)
        assert np.array_equal(out.cpu().numpy(), oD)
        assert np.array_equal(cnt.cpu().numpy(), oC)


def test_noalloc_rejects_problems_larger_than_its_scratch():
    from paper_2305_03018_gb300.morph import MORPH_E_NOMEM
    f_t = torch.zeros((1, 2048, 2048), dtype=torch.uint8, device="cuda")   # 2048*2048*64 B of planes > 64 MiB
    rc, out, cnt, status = _noalloc(f_t, 64, wl.se_flat_square(3), 0)
    assert rc == MORPH_E_NOMEM
    torch.cuda.synchronize()
    assert int(status.item()) == 12345           # nothing was queued
