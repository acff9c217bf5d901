"""CPU oracle for UTF-8 validation — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library
``libutf8gpu.so`` and its Python binding) never imports it, and this package
imports nothing from the product.

Contents
--------
* ``valid`` / ``valid_batch`` — the oracle proper: the RFC 3629 predicate of
  the paper's Section 3 (Table 1, rules a-f) as a plain decode loop in C
  (``utf8_oracle.c``).
* ``locate`` / ``locate_batch`` — where validity ends: the length of the
  longest valid prefix and the Section 3 rule (a-f, numbered 1-6) that the
  next character breaks (``RULES``), by a plain decode loop.
* ``fsm_valid`` — the Section 5 finite-state validator, an independent pin.
* ``lookup_aid`` — the Section 6 ``lookup`` steps written out plainly in
  numpy (Table 7 pattern sets -> three nibble tables, Fig. 1 classification,
  the 3-4 byte check, the end-of-stream check), used to pin the reading of
  Tables 7 and 8 and the per-byte intermediates of the GPU path.

Every function here is pinned by ``tests/test_oracle_pins.py`` against values
the paper prints, closed-form counts, Python's own strict UTF-8 codec and
brute force; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "utf8_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_libs: dict[int, ctypes.CDLL] = {}


def lib_path(mutant: int = 0) -> str:
    name = "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so"
    return os.path.join(_BUILD, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compiles the C oracle with gcc (host code only; no CUDA)."""
    out = lib_path(mutant)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = f"{out}.{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", f"-DORACLE_MUTANT={mutant}",
           "-o", tmp, _SRC, "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _load(mutant: int = 0) -> ctypes.CDLL:
    with _lock:
        if mutant in _libs:
            return _libs[mutant]
        lib = ctypes.CDLL(build(mutant))
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_valid.argtypes = [u8p, ctypes.c_size_t]
        lib.oracle_valid.restype = ctypes.c_int
        lib.oracle_fsm_valid.argtypes = [u8p, ctypes.c_size_t]
        lib.oracle_fsm_valid.restype = ctypes.c_int
        lib.oracle_valid_batch.argtypes = [u8p, i64p, ctypes.c_int64, u8p, ctypes.c_int]
        lib.oracle_valid_batch.restype = None
        lib.oracle_count_valid.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.oracle_count_valid.restype = ctypes.c_int64
        lib.oracle_valid_all.argtypes = [ctypes.c_int, u8p, ctypes.c_int]
        lib.oracle_valid_all.restype = None
        lib.oracle_class_disagreements.argtypes = [u8p, ctypes.c_int, ctypes.c_int]
        lib.oracle_class_disagreements.restype = ctypes.c_int64
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.oracle_locate.argtypes = [u8p, ctypes.c_size_t, i32p]
        lib.oracle_locate.restype = ctypes.c_int64
        lib.oracle_locate_batch.argtypes = [u8p, i64p, ctypes.c_int64, i64p, i32p, ctypes.c_int]
        lib.oracle_locate_batch.restype = None
        _libs[mutant] = lib
        return lib


def _as_u8(buf) -> np.ndarray:
    if isinstance(buf, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(buf), dtype=np.uint8)
    a = np.ascontiguousarray(buf)
    if a.dtype != np.uint8:
        raise TypeError("expected uint8 data")
    return a.reshape(-1)


def _ptr(a: np.ndarray, ctype=ctypes.c_uint8):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def valid(buf, mutant: int = 0) -> bool:
    """RFC 3629 validity of one buffer (the oracle)."""
    a = _as_u8(buf)
    if a.size == 0:
        a = np.zeros(1, dtype=np.uint8)  # valid pointer; length 0 below
        return bool(_load(mutant).oracle_valid(_ptr(a), 0))
    return bool(_load(mutant).oracle_valid(_ptr(a), a.size))


def fsm_valid(buf, mutant: int = 0) -> bool:
    """The Section 5 finite-state validator (an independent pin)."""
    a = _as_u8(buf)
    if a.size == 0:
        return True
    return bool(_load(mutant).oracle_fsm_valid(_ptr(a), a.size))


def valid_batch(data, offsets, threads: int = 1, mutant: int = 0) -> np.ndarray:
    """One uint8 flag per string k = data[offsets[k]:offsets[k+1]]."""
    d = _as_u8(data)
    o = np.ascontiguousarray(offsets, dtype=np.int64)
    count = o.size - 1
    out = np.empty(max(count, 0), dtype=np.uint8)
    if count <= 0:
        return out
    if o[0] < 0 or o[-1] > d.size or np.any(np.diff(o) < 0):
        raise ValueError("offsets must be non-decreasing and within the data")
    if d.size == 0:
        d = np.zeros(1, dtype=np.uint8)
    _load(mutant).oracle_valid_batch(_ptr(d), _ptr(o, ctypes.c_int64), count,
                                     _ptr(out), int(threads))
    return out


def count_valid(length: int, lead_min: int = 0, which: int = 0, mutant: int = 0) -> int:
    """Number of valid strings among all byte strings of ``length`` bytes
    whose first byte is >= ``lead_min`` (which=0: oracle, 1: FSM)."""
    return int(_load(mutant).oracle_count_valid(length, lead_min, which))


def valid_all(length: int, which: int = 0, mutant: int = 0) -> np.ndarray:
    """Validity of every byte string of ``length`` (1..3) bytes, indexed by the
    string read as a little-endian integer."""
    out = np.empty(256 ** length, dtype=np.uint8)
    _load(mutant).oracle_valid_all(length, _ptr(out), which)
    return out


def class_disagreements(reps, max_len: int, mutant: int = 0) -> int:
    """Decode oracle vs FSM over every class string up to ``max_len``."""
    r = _as_u8(reps)
    return int(_load(mutant).oracle_class_disagreements(_ptr(r), r.size, max_len))


# Section 3's rules, numbered as the paper letters them (0: valid).
RULES = {0: "valid", 1: "a: 5+ byte", 2: "b: too short", 3: "c: too long", 4: "d: overlong",
         5: "e: too large", 6: "f: surrogate"}


def locate(buf, mutant: int = 0) -> tuple[int, int]:
    """(length of the longest valid prefix, rule 0-6 broken by the next
    character); (len(buf), 0) for valid input."""
    a = _as_u8(buf)
    rule = ctypes.c_int32(-1)
    if a.size == 0:
        a = np.zeros(1, dtype=np.uint8)
        pos = _load(mutant).oracle_locate(_ptr(a), 0, ctypes.byref(rule))
    else:
        pos = _load(mutant).oracle_locate(_ptr(a), a.size, ctypes.byref(rule))
    return int(pos), int(rule.value)


def locate_batch(data, offsets, threads: int = 1, mutant: int = 0):
    """Per string k = data[offsets[k]:offsets[k+1]]: (positions relative to
    the string's start as int64, rules as int32)."""
    d = _as_u8(data)
    o = np.ascontiguousarray(offsets, dtype=np.int64)
    count = max(o.size - 1, 0)
    pos = np.empty(count, dtype=np.int64)
    rule = np.empty(count, dtype=np.int32)
    if count == 0:
        return pos, rule
    if o[0] < 0 or o[-1] > d.size or np.any(np.diff(o) < 0):
        raise ValueError("offsets must be non-decreasing and within the data")
    if d.size == 0:
        d = np.zeros(1, dtype=np.uint8)
    _load(mutant).oracle_locate_batch(_ptr(d), _ptr(o, ctypes.c_int64), count,
                                      _ptr(pos, ctypes.c_int64), _ptr(rule, ctypes.c_int32),
                                      int(threads))
    return pos, rule
