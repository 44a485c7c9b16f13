"""Peaks measured on the device the bench runs on, for the roofline fractions
that the measured HBM copy and BF16 GEMM figures do not cover:

* FP32 FMA: the library's own microkernel (tqs_measure_fp32_peak), the
  denominator of the ALU-bound fractions (FP32 gate arithmetic);
* TF32 tensor: cuBLAS through torch.matmul on FP32 operands with TF32
  allowed, 8192^3 (2 N^3 flops), best of 10 launches (burst) and back to back
  for about two seconds (sustained): the denominator of the TF32x3 chain;
* the SM count and L2 size of the device.
"""
from __future__ import annotations

import time


def measure(B, torch, tf32_n: int = 8192, sustained_s: float = 2.0) -> dict:
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    out = {"sms": props.multi_processor_count,
           "l2_bytes": getattr(props, "L2_cache_size", None)}
    B.tqs_measure_fp32_peak(2000)  # warm
    best = 0.0
    for _ in range(3):
        t, _ = B.tqs_measure_fp32_peak(20000)
        best = max(best, t)
    out["fp32_fma_tflops"] = best
    out["fp32_fma_how"] = ("tqs_measure_fp32_peak: 8 blocks x 256 threads per SM, 8 independent "
                           "FMA chains per thread, best of 3 launches")
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        a = torch.randn(tf32_n, tf32_n, device="cuda", dtype=torch.float32)
        b = torch.randn(tf32_n, tf32_n, device="cuda", dtype=torch.float32)
        c = torch.empty(tf32_n, tf32_n, device="cuda", dtype=torch.float32)
        for _ in range(3):
            torch.matmul(a, b, out=c)
        torch.cuda.synchronize()
        flops = 2.0 * tf32_n ** 3
        burst = 0.0
        for _ in range(10):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            torch.matmul(a, b, out=c)
            e.record()
            torch.cuda.synchronize()
            burst = max(burst, flops / (s.elapsed_time(e) * 1e-3) / 1e12)
        k = 0
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        s.record()
        while time.perf_counter() - t0 < sustained_s:
            for _ in range(8):
                torch.matmul(a, b, out=c)
            k += 8
            torch.cuda.synchronize()
        e.record()
        torch.cuda.synchronize()
        sustained = flops * k / (s.elapsed_time(e) * 1e-3) / 1e12
        del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    torch.cuda.empty_cache()
    out["tf32_tflops"] = burst
    out["tf32_tflops_sustained"] = sustained
    out["tf32_how"] = (f"torch.matmul FP32 {tf32_n}^3 with TF32 allowed (cuBLAS), best of 10 "
                       f"(burst) and back to back for {sustained_s:.0f} s (sustained)")
    return out
