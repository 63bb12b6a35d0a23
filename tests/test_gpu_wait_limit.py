"""The bounded-wait failure path of the FP8 tensor-core kernel, on the GPU.

Every mbarrier wait of k_direct_fp8 gives up after a limit (4 s by default).
With a limit of 2 microseconds -- far shorter than the tensor-core work of one
unit, which the epilogue must wait for -- a wait is bound to give up: the
kernel raises the device error word, lets its issued copies and MMAs finish,
frees its tensor memory and returns.  The test checks the reported status
(MORPH_E_TIMEOUT, read by morph_stream_check), then that the same context and
the CUDA context keep working and give exact results.  Nothing here faults,
traps or hangs: the path only returns early.  The abort and drain order itself
is checked on the CPU in test_pipeline_protocol.py.
"""
import numpy as np
import pytest

import oracle
from paper_2305_03018_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_short_wait_limit_reports_timeout_and_the_context_stays_usable():
    from paper_2305_03018_gb300.morph import MORPH_E_TIMEOUT, Context, MorphError
    ctx = Context(0)                     # a context of its own: its error word and limit are not shared
    try:
        g = wl.rng(901)
        f = g.integers(0, 64, size=(1, 1024, 1024)).astype(np.uint8)
        se = wl.se_flat_disk(31)
        ft = torch.from_numpy(f).cuda()
        ctx.set_wait_limit(2000)
        ctx.dilate(ft, 64, se, method="direct_fp8")
        with pytest.raises(MorphError) as ei:
            ctx.check()
        assert ei.value.status == MORPH_E_TIMEOUT
        ctx.check()                      # the error word was read and cleared
        ctx.set_wait_limit(0)            # back to the default limit
        for op in ("dilate", "erode"):
            fn = ctx.dilate if op == "dilate" else ctx.erode
            D, cD = fn(ft, 64, se, method="direct_fp8", count=True)
            ctx.check()
            ofn = oracle.dilate if op == "dilate" else oracle.erode
            rD, rC = ofn(f, 64, se.mask, se.offset, se.origin, nthreads=0)
            assert np.array_equal(D.cpu().numpy(), rD) and np.array_equal(cD.cpu().numpy(), rC), op
        assert int((ft.to(torch.int64) + 1).sum()) == int(f.astype(np.int64).sum()) + f.size
    finally:
        torch.cuda.synchronize()
        ctx.close()
