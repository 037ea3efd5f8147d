"""Arithmetic peaks of the GPU, measured with the library's own probe kernels.

``measure()`` runs ``libtsvd_probe.so`` (csrc/peak_probe.cu: FP64, FP32 and
packed-FP32 FMA streams, INT8 and BF16 ``mma.sync`` streams, dependent FP64 /
FP32 latency) plus two library GEMMs for context (``torch._int_mm`` for INT8,
``torch.matmul`` in float64), and returns the rates.  ``python -m
paper_2603_11953_gb300.peaks`` prints them as one JSON line.  These are the
FP64 / FP32 / INT8 denominators of the benchmark's roofline terms; HBM and
BF16 tensor peaks come from a device copy and a cuBLAS BF16 GEMM.
"""
from __future__ import annotations

import ctypes
import json
import os

from . import build as _build

KINDS = {"fp64_fma": 0, "fp32_fma": 1, "fp32x2_fma": 2, "int8_mma_sync": 3, "bf16_mma_sync": 4,
         "fp64_latency": 5, "fp32_latency": 6, "fp64_fma_1lane": 7, "fp64_fma_8lanes": 8,
         "fp64_fma_16lanes": 9}


def _lib():
    _build.build()
    lib = ctypes.CDLL(_build.PROBE_LIB)
    lib.tsvd_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_float)]
    lib.tsvd_probe.restype = ctypes.c_int
    return lib


def probe(kind: str, iters: int):
    """(operations, milliseconds) of one timed launch of probe `kind`."""
    ops, ms = ctypes.c_double(), ctypes.c_float()
    rc = _lib().tsvd_probe(KINDS[kind], int(iters), ctypes.byref(ops), ctypes.byref(ms))
    if rc != 0:
        raise RuntimeError(f"tsvd_probe({kind}) failed with CUDA error {rc}")
    return ops.value, ms.value


def _library_gemms():
    import torch
    out = {}
    dev = torch.device("cuda")
    a = torch.randint(-128, 127, (8192, 8192), dtype=torch.int8, device=dev)
    try:
        torch._int_mm(a, a)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            torch._int_mm(a, a)
        e1.record()
        torch.cuda.synchronize()
        out["int8_torch_int_mm_tops"] = 5 * 2 * 8192 ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12
    except Exception as exc:  # noqa: BLE001 - reported, not fatal
        out["int8_torch_int_mm_tops"] = f"unavailable: {exc.__class__.__name__}"
    d = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    d @ d
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        d @ d
    e1.record()
    torch.cuda.synchronize()
    out["fp64_torch_matmul_gflops"] = 3 * 2 * 4096 ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e9
    return out


def measure(library_gemms: bool = True) -> dict:
    res = {}
    for name, iters, unit, scale in (("fp64_fma", 2000, "fp64_gflops", 1e9), ("fp32_fma", 20000, "fp32_tflops", 1e12),
                                     ("fp32x2_fma", 20000, "fp32x2_tflops", 1e12),
                                     ("int8_mma_sync", 4000, "int8_mma_sync_tops", 1e12),
                                     ("bf16_mma_sync", 4000, "bf16_mma_sync_tflops", 1e12),
                                     ("fp64_fma_1lane", 2000, "fp64_1lane_gflops", 1e9),
                                     ("fp64_fma_8lanes", 2000, "fp64_8lanes_gflops", 1e9),
                                     ("fp64_fma_16lanes", 2000, "fp64_16lanes_gflops", 1e9)):
        ops, ms = probe(name, iters)
        res[unit] = ops / (ms * 1e-3) / scale
    res["fp64_fma_latency_cycles"] = probe("fp64_latency", 100000)[0]
    res["fp32_fma_latency_cycles"] = probe("fp32_latency", 100000)[0]
    if library_gemms:
        res.update(_library_gemms())
    res["how"] = ("own kernels (csrc/peak_probe.cu): 4 CTAs x 512 threads per SM, 8 independent chains per thread, "
                  "one warm-up launch then one timed launch (CUDA events); latency: one thread, one dependent chain "
                  "(clock64)")
    return res


if __name__ == "__main__":
    import torch
    torch.cuda.init()
    r = measure()
    r["gpu"] = torch.cuda.get_device_name(0)
    r["sms"] = torch.cuda.get_device_properties(0).multi_processor_count
    print(json.dumps(r))
