"""utf8_validate_host_noalloc, the host-memory validator for callers that
cannot allocate GPU memory while they validate (their device memory is
reserved up front by a pool or another framework, or a cudaMalloc could
synchronise the device on a latency-critical path), through the C-ABI.

Every expected value comes from the CPU oracle; the existing host entry
point, utf8_validate_host, must agree too.  Collected last, so that a run
stopping at the first failure has run every other test first; it passes alone
in a fresh process and after the others."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

MAX = 32 << 20  # the entry point's largest input
UTF8_OK, UTF8_ERR_BUDGET = 0, 4


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2010_03090_gb300 as u
    L = u.lib()
    # the first call on a device sets it up (and may load modules): len 0 does it
    assert L.utf8_validate_host_noalloc(None, 0, None) is True
    assert L.utf8_last_error() == UTF8_OK
    return L


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _noalloc(L, a: np.ndarray) -> bool:
    got = L.utf8_validate_host_noalloc(_ptr(a), a.size, None)
    assert L.utf8_last_error() == UTF8_OK
    return bool(got)


def _inputs():
    rng = np.random.default_rng(17)
    bufs = []
    for n, model in [(1, synth.UNIFORM), (4097, synth.CJK), (1 << 20, synth.EMOJI),
                     (MAX, synth.UNIFORM), (3_000_001, synth.LATIN)]:
        b = synth.fill(n, model, seed=n)
        bufs.append(b)
        bad = b.copy()
        synth.inject_any(bad, synth.ERROR_CLASSES[n % 7], rng)
        bufs.append(bad)
    # the largest input with a truncated character in its last three bytes
    tail = synth.fill(MAX, synth.CJK, seed=5)
    tail[-3:] = np.frombuffer(synth.tail_error_bytes(5), np.uint8)
    bufs.append(tail)
    return bufs


def test_noalloc_matches_oracle_twice(lib):
    bufs = _inputs()
    want = [oracle.valid(b) for b in bufs]
    assert not all(want) and any(want)
    for _ in range(2):  # two calls in a row on the same inputs
        for b, w in zip(bufs, want):
            assert _noalloc(lib, b) == w, b.size
            assert bool(lib.utf8_validate_host(_ptr(b), b.size, None)) == w, b.size
            assert lib.utf8_last_error() == UTF8_OK


def test_noalloc_unaligned_host_pointers(lib):
    base = synth.fill(70_000, synth.UNIFORM, seed=3)
    rng = np.random.default_rng(4)
    for off in range(1, 16):
        for n in (1, 5, 4093, 65_521):
            view = base[off:off + n]
            assert view.ctypes.data % 16 == (base.ctypes.data + off) % 16
            assert _noalloc(lib, view) == oracle.valid(view), (off, n)
            bad = view.copy()
            synth.inject_any(bad, synth.ERROR_CLASSES[(off + n) % 7], rng)
            holder = np.zeros(n + off, np.uint8)
            holder[off:] = bad
            assert _noalloc(lib, holder[off:]) == oracle.valid(bad), (off, n, "bad")


def test_noalloc_stale_bytes_never_matter(lib):
    """The staging array keeps the previous call's bytes: a short input
    validated right after a long invalid one sees none of them."""
    junk = np.full(MAX, 0xFF, np.uint8)  # invalid everywhere
    assert oracle.valid(junk) is False
    cut = np.full(MAX, 0xE4, np.uint8)  # leads waiting for continuations
    for short in (np.frombuffer(b"A", np.uint8).copy(), synth.fill(1000, synth.LATIN, seed=8),
                  np.frombuffer("é".encode(), np.uint8).copy()):
        for before in (junk, cut):
            assert _noalloc(lib, before) is False
            assert oracle.valid(short) is True
            assert _noalloc(lib, short) is True, short.size


def test_noalloc_allocates_nothing(lib):
    torch = pytest.importorskip("torch")
    bufs = _inputs()[:6]
    want = [oracle.valid(b) for b in bufs]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        for b, w in zip(bufs, want):
            assert _noalloc(lib, b) == w
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_oversize(lib):
    b = np.zeros(MAX + 1, dtype=np.uint8)
    assert lib.utf8_validate_host_noalloc(_ptr(b), b.size, None) is False
    assert lib.utf8_last_error() == UTF8_ERR_BUDGET
    assert lib.utf8_validate_host_noalloc(None, 0, None) is True
    assert lib.utf8_last_error() == UTF8_OK
