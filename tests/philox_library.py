"""Philox4x32-10 from a third-party library (PyTorch's header-only host
engine, compiled here with g++), the independent implementation that pins the
oracle's generator and, through the walk, the GPU's."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    import torch
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    out_dir = tempfile.mkdtemp(prefix="philox_library_")
    so = os.path.join(out_dir, "libphilox_library.so")
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-I", inc,
                    os.path.join(_HERE, "philox_library.cpp"), "-o", so], check=True)
    lib = ctypes.CDLL(so)
    p = ctypes.POINTER(ctypes.c_uint32)
    lib.library_philox4x32_10.argtypes = [ctypes.c_int64, p, p, p]
    _lib = lib
    return lib


def philox4x32_10(ctr, key) -> np.ndarray:
    """Words (n x 4 uint32) of counters ``ctr`` (n x 4) under keys ``key``
    (n x 2, or one key of 2 words for every counter)."""
    lib = _load()
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    key = np.asarray(key, dtype=np.uint32).reshape(-1, 2)
    key = np.ascontiguousarray(np.broadcast_to(key, (ctr.shape[0], 2)))
    out = np.empty_like(ctr)
    p = ctypes.POINTER(ctypes.c_uint32)
    lib.library_philox4x32_10(ctr.shape[0], ctr.ctypes.data_as(p), key.ctypes.data_as(p),
                              out.ctypes.data_as(p))
    return out
