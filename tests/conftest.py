import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


GOLDEN = os.path.join(ROOT, "tests", "golden")


def _bwd_chunks(n, h, w, ntaps):
    """Chunks of the backward's SE-gradient partial sums: up to 1024 taps, runs of 256 M
    consecutive pixels of one image (M = 8, 4, 2, 1: the largest with four CTAs per SM of
    152); else rows x columns blocks of at most 8192 pixels."""
    npx = h * w
    if 0 < ntaps <= 1024:
        m = 8
        while m > 1 and npx * n // (256 * m) < 4 * 152:
            m //= 2
        return n * -(-npx // (256 * m))
    cb = min(w, 8192)
    rb = max(1, 8192 // cb)
    return n * -(-h // rb) * -(-w // cb)


@pytest.fixture
def bwd_chunks():
    return _bwd_chunks
