"""Measured ceilings for the bench's rooflines (libnqs_peaks.so, peaks.cu).

measure(device) returns, for one GB300:
  l2_read_gbs[size_mb]   streaming 16-byte reads over a buffer of that size,
                         repeated so that it stays resident in L2 (129 MB);
  hbm_read_gbs           the same over 4 GiB (read-only DRAM rate);
  gather8_gbs[size_mb]   independent random 8-byte loads from a table of that
                         size, in useful bytes per second (the integral
                         reads of the Slater-Condon elements have this shape);
  fma64_tflops, fma32_tflops   CUDA-core fused multiply-add rates.
Each figure is the best of three timed launch groups (CUDA events).
"""
from __future__ import annotations

import ctypes
import os

from .. import build as _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build_peaks()
        lib = ctypes.CDLL(path)
        for name in ("peaks_read", "peaks_gather8"):
            getattr(lib, name).argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.POINTER(ctypes.c_float)]
        for name in ("peaks_fma64", "peaks_fma32"):
            getattr(lib, name).argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                           ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]
        _LIB = lib
    return _LIB


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed with CUDA error {rc}")


def measure(device=0, l2_sizes_mb=(16, 32, 50, 64, 96), gather_sizes_mb=(32, 64)):
    import torch
    lib = _lib()
    dev = torch.device("cuda", device)
    torch.cuda.set_device(dev)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    st = torch.cuda.current_stream(dev).cuda_stream
    sink = torch.zeros(1 << 16, dtype=torch.float64, device=dev)
    ms = ctypes.c_float()
    out = {"n_sm": n_sm, "l2_read_gbs": {}, "gather8_gbs": {}}

    def best(fn, *args):
        t = []
        for _ in range(3):
            _check(fn(*args, 5, ctypes.c_void_p(st), ctypes.byref(ms)), fn.__name__)
            t.append(ms.value)
        return min(t)

    blocks = 8 * n_sm
    for mb in l2_sizes_mb:
        nbytes = mb << 20
        buf = torch.zeros(nbytes // 4, dtype=torch.float32, device=dev)
        passes = max(1, (4 << 30) // nbytes)
        t = best(lib.peaks_read, ctypes.c_void_p(buf.data_ptr()), nbytes, passes, blocks,
                 ctypes.c_void_p(sink.data_ptr()))
        out["l2_read_gbs"][str(mb)] = nbytes * passes / (t * 1e-3) / 1e9
        del buf
    nbytes = 4 << 30
    buf = torch.zeros(nbytes // 4, dtype=torch.float32, device=dev)
    t = best(lib.peaks_read, ctypes.c_void_p(buf.data_ptr()), nbytes, 1, blocks, ctypes.c_void_p(sink.data_ptr()))
    out["hbm_read_gbs"] = nbytes / (t * 1e-3) / 1e9
    del buf
    gblocks, loads = 16 * n_sm, 512
    for mb in gather_sizes_mb:
        words = (mb << 20) // 8
        buf = torch.zeros(words, dtype=torch.float64, device=dev)
        t = best(lib.peaks_gather8, ctypes.c_void_p(buf.data_ptr()), words, loads, gblocks,
                 ctypes.c_void_p(sink.data_ptr()))
        out["gather8_gbs"][str(mb)] = 8.0 * gblocks * 256 * loads / (t * 1e-3) / 1e9
        del buf
    iters = 8192
    for name, fn in (("fma64_tflops", lib.peaks_fma64), ("fma32_tflops", lib.peaks_fma32)):
        t = best(fn, iters, blocks, ctypes.c_void_p(sink.data_ptr()))
        out[name] = 2.0 * 8 * iters * blocks * 256 / (t * 1e-3) / 1e12
    torch.cuda.synchronize(dev)
    return out
