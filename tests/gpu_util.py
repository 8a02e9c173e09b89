"""Device-memory helpers for the GPU tests (torch for allocation, the CUDA
runtime that libdock.so already loaded for raw-pointer copies)."""
from __future__ import annotations

import ctypes as C

import numpy as np

_rt = None


def rt():
    global _rt
    if _rt is None:
        for name in ("libcudart.so.13", "libcudart.so"):
            try:
                _rt = C.CDLL(name)
                break
            except OSError:
                continue
        if _rt is None:
            raise RuntimeError("CUDA runtime library not found")
        _rt.cudaMemcpy.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]
        _rt.cudaMemcpy.restype = C.c_int
    return _rt


def d2h(ptr: int, count: int, dtype) -> np.ndarray:
    out = np.empty(count, dtype)
    if count:
        err = rt().cudaMemcpy(out.ctypes.data, C.c_void_p(ptr), out.nbytes, 2)
        if err != 0:
            raise RuntimeError("cudaMemcpy D2H failed: %d" % err)
    return out


def to_dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()
