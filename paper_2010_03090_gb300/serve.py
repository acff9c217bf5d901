"""Continuous-batching validation server: a thin binding of the C-ABI
utf8_server_* calls (the scheduler, admission and batching run in the
library's native worker thread)."""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import Utf8Error, _check, _dev, lib


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("window_min_us", ctypes.c_uint32),
                ("window_max_us", ctypes.c_uint32), ("max_batch", ctypes.c_uint32),
                ("streams", ctypes.c_uint32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "completed", "batches", "bytes",
                                               "max_admitted_bytes", "max_batch_seen")]


_bound = False


def _bind():
    global _bound
    if _bound:
        return lib()
    L = lib()
    vp, sz, i64, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int64, ctypes.c_int
    L.utf8_server_default_config.argtypes = [ctypes.POINTER(ServerConfig)]
    L.utf8_server_default_config.restype = None
    L.utf8_server_create.argtypes = [ctypes.POINTER(ServerConfig)]
    L.utf8_server_create.restype = vp
    L.utf8_server_submit.argtypes = [vp, vp, sz, ctypes.POINTER(ctypes.c_uint64)]
    L.utf8_server_submit.restype = i32
    L.utf8_server_result.argtypes = [vp, ctypes.c_uint64, i64, ctypes.POINTER(i32),
                                     ctypes.POINTER(i64)]
    L.utf8_server_result.restype = i32
    L.utf8_server_replay.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(sz),
                                     ctypes.POINTER(i64), i64, ctypes.POINTER(ctypes.c_uint8),
                                     ctypes.POINTER(i64)]
    L.utf8_server_replay.restype = i32
    L.utf8_server_stats_get.argtypes = [vp, ctypes.POINTER(ServerStats)]
    L.utf8_server_stats_get.restype = i32
    L.utf8_server_destroy.argtypes = [vp]
    L.utf8_server_destroy.restype = None
    _bound = True
    return L


def default_config() -> dict:
    c = ServerConfig()
    _bind().utf8_server_default_config(ctypes.byref(c))
    return {n: getattr(c, n) for n, _ in ServerConfig._fields_}


class Server:
    """Submit device tensors; results come back as (valid, latency_ns)."""

    def __init__(self, **config):
        L = _bind()
        c = ServerConfig()
        L.utf8_server_default_config(ctypes.byref(c))
        for k, v in config.items():
            setattr(c, k, v)
        self._h = L.utf8_server_create(ctypes.byref(c))
        if not self._h:
            raise Utf8Error(L.utf8_last_error(), "utf8_server_create")

    def submit(self, data) -> int:
        p, n = _dev(data, "uint8", "data")
        t = ctypes.c_uint64()
        _check(_bind().utf8_server_submit(self._h, p or None, n, ctypes.byref(t)),
               "utf8_server_submit")
        return t.value

    def result(self, ticket: int, timeout_us: int = -1):
        v, lat = ctypes.c_int(), ctypes.c_int64()
        _check(_bind().utf8_server_result(self._h, ticket, timeout_us, ctypes.byref(v),
                                          ctypes.byref(lat)), "utf8_server_result")
        return bool(v.value), lat.value

    def replay(self, ptrs, lens, arrival_ns):
        """ptrs: device addresses (ints), lens: sizes, arrival_ns: offsets from
        the start; returns (valid uint8[n], latency_ns int64[n])."""
        n = len(lens)
        p = np.ascontiguousarray(ptrs, dtype=np.uint64)
        ln = np.ascontiguousarray(lens, dtype=np.uint64)
        ar = np.ascontiguousarray(arrival_ns, dtype=np.int64)
        valid = np.zeros(n, dtype=np.uint8)
        lat = np.zeros(n, dtype=np.int64)
        _check(_bind().utf8_server_replay(
            self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_void_p)),
            ln.ctypes.data_as(ctypes.POINTER(ctypes.c_size_t)),
            ar.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n,
            valid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
            lat.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), "utf8_server_replay")
        return valid, lat

    def stats(self) -> dict:
        s = ServerStats()
        _bind().utf8_server_stats_get(self._h, ctypes.byref(s))
        return {n: getattr(s, n) for n, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            _bind().utf8_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
