"""Instruction-throughput probes (include/casim_peaks.h), for the rooflines of
the step kernels.  ctypes marshalling only; raises if the library is missing."""
from __future__ import annotations

import ctypes
import os

from .build import PEAKS_LIB

KINDS = {"ffma": 0, "dfma": 1, "ex2": 2, "lg2": 3, "rcp": 4, "tanh": 5, "tanh_bf16x2": 6}
_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(PEAKS_LIB):
            raise RuntimeError(f"{PEAKS_LIB} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(PEAKS_LIB)
        L.casim_peak_rate.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_double)]
        L.casim_peak_rate.restype = ctypes.c_int
        _lib = L
    return _lib


def peak_rate(kind: str, iters: int, stream=None) -> float:
    """Operations per second of `kind` over the whole GPU (one FMA = one operation)."""
    r = ctypes.c_double(0.0)
    st = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    rc = lib().casim_peak_rate(KINDS[kind], iters, ctypes.c_void_p(st), ctypes.byref(r))
    if rc != 0:
        raise RuntimeError(f"casim_peak_rate({kind}) failed: {rc}")
    return r.value
