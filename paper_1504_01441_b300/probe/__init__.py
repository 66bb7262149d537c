"""Measurement aid of the benchmark: the integer dot-product rate probe.

Built as libhdrreg_probe.so (``build.build()`` compiles it beside the registration
library) and loaded only by the benchmark and its test; it is not part of the
registration library's C ABI.
"""
import ctypes as C
import os

LIB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libhdrreg_probe.so")
_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: run paper_1504_01441_b300.build.build()")
        _lib = C.CDLL(LIB)
        _lib.hdrreg_probe_dp4a.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p]
        _lib.hdrreg_probe_dp4a.restype = C.c_int
    return _lib


def probe_dp4a(blocks: int, iters: int, sink, stream=None) -> int:
    """Enqueue the probe (``sink``: a CUDA int32 tensor of one element) on ``stream`` (a
    torch stream; the current stream when None); -> the number of __dp4a it issues."""
    import torch
    st = C.c_void_p((stream if stream is not None else torch.cuda.current_stream()).cuda_stream)
    rc = lib().hdrreg_probe_dp4a(int(blocks), int(iters), C.c_void_p(sink.data_ptr()), st)
    if rc != 0:
        raise RuntimeError(f"hdrreg_probe_dp4a({blocks}, {iters}) returned {rc}")
    return blocks * 256 * iters * 8
