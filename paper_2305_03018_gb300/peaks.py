"""Measured arithmetic peaks of this GPU for the rooflines the library reports.

Library GEMMs stand in for each unit's peak: FP8 E4M3 dense (cuBLASLt through
``torch._scaled_mm``), FP32 without tensor cores (SGEMM with TF32 disabled,
i.e. FMA-pipe bound) and FP64 (DGEMM).  Each is timed with CUDA events as a
burst (best of 10) and as a loop of about 2 s (sustained).

    python -m paper_2305_03018_gb300.peaks      # prints one JSON line
"""
from __future__ import annotations

import json
import time


def _time_gemm(fn, flop, seconds=2.0):
    import torch
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(10):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    reps = max(1, int(seconds * 1e3 / best))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    sus = e0.elapsed_time(e1) / reps
    return flop / (best * 1e-3) / 1e12, flop / (sus * 1e-3) / 1e12


def measure() -> dict:
    import torch
    out = {"gpu": torch.cuda.get_device_name(), "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    n = 8192
    a = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
    b = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn).t()
    one = torch.ones((), device="cuda")
    try:
        burst, sus = _time_gemm(lambda: torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16),
                                2.0 * n ** 3)
        out["fp8_e4m3_tflops"] = burst
        out["fp8_e4m3_tflops_sustained"] = sus
    except Exception as e:                         # keep the other peaks if FP8 GEMM is unavailable
        out["fp8_error"] = str(e)[:200]
    del a, b
    torch.backends.cuda.matmul.allow_tf32 = False
    n = 8192
    x = torch.randn(n, n, device="cuda", dtype=torch.float32)
    y = torch.randn(n, n, device="cuda", dtype=torch.float32)
    out["fp32_tflops"], out["fp32_tflops_sustained"] = _time_gemm(lambda: x @ y, 2.0 * n ** 3)
    del x, y
    n = 4096
    x = torch.randn(n, n, device="cuda", dtype=torch.float64)
    y = torch.randn(n, n, device="cuda", dtype=torch.float64)
    out["fp64_tflops"], out["fp64_tflops_sustained"] = _time_gemm(lambda: x @ y, 2.0 * n ** 3)
    out["how"] = ("CUDA events; burst = best of 10, sustained = ~2 s loop; FP8 via torch._scaled_mm "
                  "(E4M3 x E4M3 -> bf16, 8192^3), FP32 SGEMM with TF32 off (8192^3), FP64 DGEMM (4096^3)")
    return out


if __name__ == "__main__":
    print(json.dumps(measure()), flush=True)
