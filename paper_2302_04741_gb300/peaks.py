"""Measured arithmetic rates of the current GPU (csrc/alu_peaks.cu): the
ceiling of the FP64 step, which GB300's FP64 units, not HBM, bound.

    python -m paper_2302_04741_gb300.peaks      # prints the rates as JSON
"""
import ctypes
import json
import os
import subprocess

from paper_2302_04741_gb300 import build as B

LIB = os.path.join(B.BUILD, "libalu_peaks.so")
SRC = os.path.join(B.CSRC, "alu_peaks.cu")
KINDS = {"dfma": 0, "dadd": 1, "ffma": 2, "f64_f32_convert": 3, "int32": 5, "ffma_packed_f32x2": 6,
         "f32_f16_convert": 7}


def build():
    os.makedirs(B.BUILD, exist_ok=True)
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call([B._nvcc()] + B.ARCH + ["-O3", "-shared", "-Xcompiler", "-fPIC",
                                                     "-cudart", "shared", "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


def rates(reps=5):
    """Operations per second of each probe (an FMA is one operation)."""
    L = ctypes.CDLL(build())
    L.alu_probe.restype = ctypes.c_double
    L.alu_probe.argtypes = [ctypes.c_int, ctypes.c_int]
    return {k: L.alu_probe(v, reps) for k, v in KINDS.items()}


if __name__ == "__main__":
    r = rates()
    print(json.dumps({k: v / 1e12 for k, v in r.items()} | {"unit": "Tops/s (FMA = 1 op)"}, indent=1))
