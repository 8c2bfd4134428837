"""Measured issue rates of the FP64, FP32 FMA and integer ALU pipes of this GPU (thread
operations per second), from the chain probes in csrc/peaks.cu (libpeaks.so). They are
the denominators of the FP64 and integer-pipe rooflines: the driver's peak file carries an
HBM copy and a bf16 GEMM figure only.

    python -m paper_1811_08282_gb300.peaks
"""
from __future__ import annotations

import ctypes
import json

from . import build

KINDS = {"fp64_fma": (0, 4096), "fp32_fma": (1, 65536), "int_alu": (2, 65536)}


def measure() -> dict:
    """{kind: thread operations per second} for the three probes (best of three)."""
    lib = ctypes.CDLL(build.build_peaks())
    lib.pk_rate.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.pk_rate.restype = ctypes.c_double
    out = {}
    for name, (kind, iters) in KINDS.items():
        rates = [lib.pk_rate(kind, iters) for _ in range(3)]
        if min(rates) < 0:
            raise RuntimeError(f"peak probe {name} failed")
        out[name] = max(rates)
    return out


if __name__ == "__main__":
    import torch
    torch.cuda.init()
    r = measure()
    print(json.dumps({k: v / 1e9 for k, v in r.items()} | {"unit": "G thread operations/s"}))
