"""Seeded synthetic UTF-8 inputs (shared input source for tests and bench).

Holds no validation arithmetic.  ``synth.c`` fills buffers with valid UTF-8
from a counter-based SplitMix64 stream; this wrapper adds error injection
(in place, length preserving, at a character boundary) and the workload
recipes: the 1 MiB buffer with seven corrupted copies, the 1 GiB content
variants, the 1M-string log-normal batch, the 20k-string Pareto batch and
the serving request mix.  Expected validity always comes from the oracle.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libsynth.so")
_lock = threading.Lock()
_lib = None

ASCII, LATIN, CJK, EMOJI, UNIFORM, RAND12, RAND13 = range(7)
MODEL_NAMES = {"ascii": ASCII, "latin": LATIN, "cjk": CJK, "emoji": EMOJI,
               "uniform": UNIFORM, "rand12": RAND12, "rand13": RAND13}

ERROR_CLASSES = ("too_short", "too_long", "overlong", "too_large", "surrogate",
                 "stray", "truncated")

SEED_BASE = 20100309


def build(force: bool = False) -> str:
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = f"{_LIB}.{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC,
                    "-lpthread"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p = ctypes.POINTER(ctypes.c_uint8)
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.synth_fill.argtypes = [u8p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int]
            lib.synth_fill_strings.argtypes = [u8p, i64p, ctypes.c_int64, u8p, ctypes.c_int,
                                               ctypes.c_uint64, ctypes.c_int64, ctypes.c_int,
                                               i64p]
            _lib = lib
    return _lib


def default_threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def fill_strings(offsets, model=UNIFORM, seed: int = SEED_BASE, threads: int | None = None,
                 seg: int = 1 << 20, out: np.ndarray | None = None) -> np.ndarray:
    """Valid UTF-8 for every string of ``offsets``; ``model`` is one content
    model for all strings or a uint8 array with one model per string."""
    o = np.ascontiguousarray(offsets, dtype=np.int64)
    count = o.size - 1
    total = int(o[-1]) if o.size else 0
    data = out if out is not None else np.empty(max(total, 1), dtype=np.uint8)
    if count <= 0 or total == 0:
        return data[:total]
    models = None
    mval = 0
    if np.ndim(model) == 0:
        mval = int(model)
    else:
        models = np.ascontiguousarray(model, dtype=np.uint8)
        assert models.size == count
    scratch = np.empty(count + 1, dtype=np.int64)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    i64p = ctypes.POINTER(ctypes.c_int64)
    _load().synth_fill_strings(
        data.ctypes.data_as(u8p), o.ctypes.data_as(i64p), count,
        models.ctypes.data_as(u8p) if models is not None else None, mval,
        ctypes.c_uint64(seed & (2 ** 64 - 1)), seg, threads or default_threads(),
        scratch.ctypes.data_as(i64p))
    return data[:total]


def fill(n: int, model=UNIFORM, seed: int = SEED_BASE, threads: int | None = None,
         out: np.ndarray | None = None) -> np.ndarray:
    """Exactly ``n`` bytes of valid UTF-8 (one buffer, 1 MiB segments)."""
    return fill_strings(np.array([0, n], dtype=np.int64), model, seed, threads, out=out)


# ---------------------------------------------------------------------------
# error injection (in place, length preserving)
# ---------------------------------------------------------------------------
_PREFIX = {1: b"\xc3", 2: b"\xe9\x8f", 3: b"\xf0\x9f\x98"}


def _is_start(b: int) -> bool:
    return (b & 0xC0) != 0x80


def _char_len(b: int) -> int:
    return 1 if b < 0x80 else 2 if b < 0xE0 else 3 if b < 0xF0 else 4


def _run_of(buf, c, hi, length):
    """True if whole characters starting at c cover exactly `length` bytes."""
    total = 0
    while total < length and c + total < hi:
        total += _char_len(int(buf[c + total]))
    return total == length and c + total <= hi


def inject(buf: np.ndarray, kind: str, rng: np.random.Generator, lo: int = 0,
           hi: int | None = None, at: int | None = None, scan: int = 1 << 16):
    """Injects one error of class ``kind`` into valid text buf[lo:hi].

    The search starts at ``at`` (or a random offset) and walks forward to the
    first character boundary where the class fits.  Returns the first
    modified offset, or None if the class does not fit in the region."""
    hi = buf.size if hi is None else hi
    if hi <= lo:
        return None
    r = lambda n: int(rng.integers(0, n))  # noqa: E731
    if kind == "truncated":
        t = 1 + r(3)
        for length in range(t, min(t + 4, hi - lo + 1)):
            start = hi - length
            if start >= lo and _is_start(int(buf[start])) and _run_of(buf, start, hi, length):
                buf[start:hi] = np.frombuffer(b"x" * (length - t) + _PREFIX[t], dtype=np.uint8)
                return hi - t
        return None
    start = at if at is not None else lo + r(hi - lo)
    start = min(max(start, lo), hi - 1)
    for step in range(min(scan, hi - lo)):
        c = lo + (start - lo + step) % (hi - lo)
        b = int(buf[c])
        if not _is_start(b):
            continue
        k = _char_len(b)
        if c + k > hi:
            continue
        if kind == "too_short" and k >= 2:
            buf[c + k - 1] = ord("A")
            return c + k - 1
        if kind == "too_long" and k >= 2 and c + k < hi and int(buf[c + k]) < 0x80:
            buf[c + k] = 0x80 + r(64)
            return c + k
        if kind == "overlong" and k >= 2:
            if k == 2:
                buf[c] = 0xC0 + r(2)
            elif k == 3:
                buf[c], buf[c + 1] = 0xE0, 0x80 + r(32)
            else:
                buf[c], buf[c + 1] = 0xF0, 0x80 + r(16)
            return c
        if kind == "too_large":
            if k == 4:
                if r(2):
                    buf[c], buf[c + 1] = 0xF4, 0x90 + r(48)
                else:
                    buf[c] = 0xF5 + r(11)
                return c
            if step > 4096 and _run_of(buf, c, hi, 4):
                buf[c:c + 4] = [0xF4, 0x90 + r(48), 0x80 + r(64), 0x80 + r(64)]
                return c
        if kind == "surrogate":
            if k == 3:
                buf[c], buf[c + 1] = 0xED, 0xA0 + r(32)
                return c
            if step > 4096 and _run_of(buf, c, hi, 3):
                buf[c:c + 3] = [0xED, 0xA0 + r(32), 0x80 + r(64)]
                return c
        if kind == "stray" and k == 1 and (c == lo or int(buf[c - 1]) < 0x80):
            buf[c] = 0x80 + r(64)
            return c
    if kind in ("too_large", "surrogate"):
        # no suitable character near the start: take any run of whole chars
        need = 4 if kind == "too_large" else 3
        for c in range(lo, hi - need + 1):
            if _is_start(int(buf[c])) and _run_of(buf, c, hi, need):
                if need == 4:
                    buf[c:c + 4] = [0xF4, 0x90 + r(48), 0x80 + r(64), 0x80 + r(64)]
                else:
                    buf[c:c + 3] = [0xED, 0xA0 + r(32), 0x80 + r(64)]
                return c
    return None


def inject_any(buf, kind, rng, lo=0, hi=None, at=None):
    """``inject`` with the closest feasible class for short regions: a lone
    continuation (stray) or a lone lead byte at the end (truncated)."""
    hi = buf.size if hi is None else hi
    pos = inject(buf, kind, rng, lo, hi, at)
    if pos is None and hi > lo:
        pos = inject(buf, "stray", rng, lo, hi, at)
    if pos is None and hi > lo:
        pos = inject(buf, "truncated", rng, lo, hi)
    if pos is None and hi > lo:
        buf[lo] = 0x80 + int(rng.integers(0, 64))
        pos = lo
    return pos


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def workload_1mib(seed: int = SEED_BASE):
    """1 MiB of the uniform 1-4 byte mix plus seven corrupted copies, one per
    error class.  Returns (list of 8 arrays, list of labels)."""
    n = 1 << 20
    base = fill(n, UNIFORM, seed)
    bufs, labels = [base], ["valid"]
    rng = np.random.default_rng(seed)
    for kind in ERROR_CLASSES:
        b = base.copy()
        pos = inject(b, kind, rng)
        assert pos is not None, kind
        bufs.append(b)
        labels.append(kind)
    return bufs, labels


VARIANTS_1GIB = ("ascii", "latin", "cjk", "emoji", "uniform")


def fill_variant(n: int, name: str, seed: int = SEED_BASE, threads: int | None = None,
                 out: np.ndarray | None = None) -> np.ndarray:
    """One content variant of exactly n bytes whose last 3 bytes are ASCII,
    so a character ends at n - 3 (room for a tail error)."""
    buf = fill(n - 3, MODEL_NAMES[name], seed, threads,
               out=out[:n - 3] if out is not None else None)
    full = out if out is not None else np.empty(n, dtype=np.uint8)
    if out is None:
        full[:n - 3] = buf
    full[n - 3:] = np.frombuffer(b"xyz", dtype=np.uint8)
    return full


def tail_error_bytes(seed: int) -> bytes:
    """The last 3 bytes of a tail-error copy: ASCII then a truncated prefix of
    1-3 bytes chosen by the seed."""
    t = 1 + int(np.random.default_rng(seed).integers(0, 3))
    return b"x" * (3 - t) + _PREFIX[t]


def lognormal_lengths(count: int, median: float, total: int, lo: int, hi: int, seed: int):
    """Log-normal lengths with the given median, clipped to [lo, hi]; sigma is
    found by bisection so that the sum is close to ``total``."""
    z = np.random.default_rng(seed).standard_normal(count)

    def lengths(sigma):
        return np.clip(np.rint(median * np.exp(sigma * z)), lo, hi).astype(np.int64)

    a, b = 0.0, 4.0
    for _ in range(60):
        mid = (a + b) / 2
        if lengths(mid).sum() < total:
            a = mid
        else:
            b = mid
    return lengths((a + b) / 2), (a + b) / 2


def pareto_lengths(count: int, alpha: float, total: int, lo: int, hi: int, seed: int):
    """Pareto(alpha) shapes scaled by s (bisection) so that the sum of
    clip(s * L, lo, hi) is close to ``total``."""
    u = np.random.default_rng(seed).random(count)
    shape = (1.0 - u) ** (-1.0 / alpha)

    def lengths(s):
        return np.clip(np.rint(s * shape), lo, hi).astype(np.int64)

    a, b = 0.0, float(hi)
    for _ in range(100):
        mid = (a + b) / 2
        if lengths(mid).sum() < total:
            a = mid
        else:
            b = mid
    return lengths((a + b) / 2), (a + b) / 2


def offsets_of(lengths) -> np.ndarray:
    o = np.zeros(len(lengths) + 1, dtype=np.int64)
    o[1:] = np.cumsum(lengths)
    return o


def corrupt_strings(data, offsets, fraction: float, seed: int, at_boundaries=None):
    """Corrupts a seeded ``fraction`` of the strings with a uniformly chosen
    error class.  ``at_boundaries`` (a list of byte periods) places each error
    within 3 bytes before a multiple of a period inside the string.  Returns
    the indices of the corrupted strings."""
    rng = np.random.default_rng(seed)
    count = offsets.size - 1
    k = max(1, int(round(count * fraction)))
    idx = np.sort(rng.choice(count, size=k, replace=False))
    for i in idx:
        lo, hi = int(offsets[i]), int(offsets[i + 1])
        if hi <= lo:
            continue
        kind = ERROR_CLASSES[int(rng.integers(0, len(ERROR_CLASSES)))]
        at = None
        if at_boundaries:
            period = at_boundaries[int(rng.integers(0, len(at_boundaries)))]
            nb = (hi - lo) // period
            if nb >= 1:
                at = lo + period * int(rng.integers(1, nb + 1)) - int(rng.integers(0, 4))
                kind = ("too_short", "too_long", "overlong", "surrogate",
                        "too_large", "stray")[int(rng.integers(0, 6))]
        inject_any(data, kind, rng, lo, hi, at)
    return idx


def workload_batch_1m(seed: int = SEED_BASE + 2000, count: int = 1_000_000,
                      total: int = 512 << 20, threads: int | None = None):
    """1M strings, log-normal lengths (median 200 B, clipped 1 B..64 KiB,
    about 512 MiB in all), uniform-mix content, 1% corrupted."""
    lengths, _ = lognormal_lengths(count, 200.0, total, 1, 65536, seed)
    offsets = offsets_of(lengths)
    data = fill_strings(offsets, UNIFORM, seed, threads)
    bad = corrupt_strings(data, offsets, 0.01, seed + 1)
    return data, offsets, bad


def workload_heavy_skew(seed: int = SEED_BASE + 3000, count: int = 20_000,
                        total: int = 4 << 30, boundaries=(2048, 65536),
                        threads: int | None = None):
    """20k strings, Pareto(1.1) lengths scaled to about 4 GiB in all (8 B ..
    256 MiB), CJK and emoji content alternating, 0.1% corrupted with errors
    placed just before multiples of the given byte periods."""
    lengths, _ = pareto_lengths(count, 1.1, total, 8, 256 << 20, seed)
    offsets = offsets_of(lengths)
    models = np.where(np.arange(count) % 2 == 0, CJK, EMOJI).astype(np.uint8)
    data = fill_strings(offsets, models, seed, threads)
    bad = corrupt_strings(data, offsets, 0.001, seed + 1, at_boundaries=list(boundaries))
    return data, offsets, bad


def serving_requests(seed: int = SEED_BASE + 4000, duration_s: float = 10.0,
                     rate: float = 50_000.0, lo: int = 64, hi: int = 16 << 20):
    """Poisson arrival times and log-uniform sizes of a serving run."""
    rng = np.random.default_rng(seed)
    n = int(rng.poisson(rate * duration_s))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n))
    sizes = np.exp(rng.uniform(math.log(lo), math.log(hi), n)).astype(np.int64)
    return arrivals, sizes


def serving_pool(count: int = 2048, lo: int = 64, hi: int = 16 << 20,
                 invalid_fraction: float = 0.005, seed: int = SEED_BASE + 4000,
                 threads: int | None = None):
    """Request payloads for a serving run: ``count`` strings with log-uniform
    sizes in [lo, hi], mixed content, a seeded fraction corrupted.  Requests
    draw payloads uniformly, so their sizes are log-uniform too.  Returns
    (data, offsets, indices of the corrupted payloads)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(lo), math.log(hi), count)).astype(np.int64)
    offsets = offsets_of(sizes)
    data = fill_strings(offsets, UNIFORM, seed, threads)
    bad = corrupt_strings(data, offsets, invalid_fraction, seed + 1)
    return data, offsets, bad


def poisson_arrivals_ns(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival offsets (ns from the start) of a Poisson process."""
    rng = np.random.default_rng(seed)
    return (np.cumsum(rng.exponential(1.0 / rate, count)) * 1e9).astype(np.int64)
