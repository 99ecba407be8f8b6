"""Measured FP32 and FP64 FMA throughput of the current GPU (libnphc_peak.so, built from
csrc/alu_peak.cu): the denominators of the trackers' ALU roofline."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
PEAK_LIB = os.path.join(_HERE, "_build", "libnphc_peak.so")
_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(PEAK_LIB):
            raise RuntimeError(f"{PEAK_LIB} not built; run paper_1104_5497_gb300.build.build()")
        L = ctypes.CDLL(PEAK_LIB)
        L.nphc_alu_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)]
        L.nphc_alu_peak.restype = ctypes.c_int
        _lib = L
    return _lib


def alu_peak(precision: int, blocks_per_sm: int = 4, iters: int | None = None) -> dict:
    """FMA throughput (TFLOP/s, 2 flops per FMA) for precision 32 or 64: the best of three
    launches of independent FMA chains over every SM."""
    if iters is None:
        iters = 20000 if precision == 32 else 1500
    best = None
    for _ in range(3):
        t, ms = ctypes.c_double(), ctypes.c_float()
        if _load().nphc_alu_peak(int(precision), int(blocks_per_sm), int(iters), ctypes.byref(t),
                                 ctypes.byref(ms)):
            raise RuntimeError(f"nphc_alu_peak({precision}) failed")
        if best is None or t.value > best["tflops"]:
            best = {"tflops": t.value, "ms": float(ms.value)}
    best.update(precision=precision, blocks_per_sm=blocks_per_sm, iters=iters)
    return best
