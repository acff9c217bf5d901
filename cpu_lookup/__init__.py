"""The paper's `lookup` validator on the host CPU (16-byte vectors; tbl/ext on
Arm), a CPU baseline for context -- used only by the tests and the benchmark.

It is not the oracle (the oracle is the plain decode loop of Section 3 in
``oracle/``) and not a fallback of the GPU library, which never loads it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lookup_vec.c")
_LIB = os.path.join(_HERE, "_build", "libcpulookup.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the library with gcc (-O3, no -march: the same source and
    results on x86-64 and aarch64)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = f"{_LIB}.{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O3", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lpthread"],
                   check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p, i64p = ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_int64)
            lib.cpu_lookup_valid.argtypes = [u8p, ctypes.c_size_t]
            lib.cpu_lookup_valid.restype = ctypes.c_int
            lib.cpu_lookup_valid_batch.argtypes = [u8p, i64p, ctypes.c_int64, u8p, ctypes.c_int]
            lib.cpu_lookup_valid_batch.restype = None
            _lib = lib
        return _lib


def _u8(buf) -> np.ndarray:
    if isinstance(buf, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(buf), dtype=np.uint8)
    a = np.ascontiguousarray(buf)
    if a.dtype != np.uint8:
        raise TypeError("expected uint8 data")
    return a.reshape(-1)


def valid(buf) -> bool:
    a = _u8(buf)
    if a.size == 0:
        return True
    return bool(_load().cpu_lookup_valid(a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), a.size))


def valid_batch(data, offsets, threads: int = 1) -> np.ndarray:
    d = _u8(data)
    o = np.ascontiguousarray(offsets, dtype=np.int64)
    count = max(o.size - 1, 0)
    out = np.empty(count, dtype=np.uint8)
    if count == 0:
        return out
    if o[0] < 0 or o[-1] > d.size or np.any(np.diff(o) < 0):
        raise ValueError("offsets must be non-decreasing and within the data")
    if d.size == 0:
        d = np.zeros(1, dtype=np.uint8)
    _load().cpu_lookup_valid_batch(d.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                   o.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), count,
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                   int(threads))
    return out
