"""Measurement helpers for the bench, outside liblqcd and its ABI.

``fma_probe(sink, prec, iters, blocks, stream=None)`` runs the FMA-chain probe
of ``fma_probe.cu`` (libfma_probe.so, built by ``paper_1512_03487_gb300/build.py``
beside liblqcd.so): the FP64 (prec 0) or FP32 (prec 1) FMA rate that ALU-bound
kernels are quoted against.
"""
from __future__ import annotations

import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "libfma_probe.so")

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built: run paper_1512_03487_gb300/build.py")
        _lib = C.CDLL(LIB_PATH)
        _lib.fma_probe.restype = C.c_int
        _lib.fma_probe.argtypes = [C.c_void_p, C.c_int, C.c_int64, C.c_int, C.c_void_p]
    return _lib


def fma_probe(sink, prec: int, iters: int, blocks: int, stream=None) -> None:
    ptr = sink.data_ptr() if hasattr(sink, "data_ptr") else sink
    st = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)
    rc = lib().fma_probe(C.c_void_p(ptr), int(prec), int(iters), int(blocks), C.c_void_p(st) if st else None)
    if rc != 0:
        raise RuntimeError(f"fma_probe failed with status {rc}")
