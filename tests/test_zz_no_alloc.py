"""utf8_validate_host_noalloc (the entry point for callers that cannot
allocate GPU memory) against utf8_validate_host, through the C-ABI.

Collected last so that a run stopping at the first failure has run every
other test first.  Passes alone in a fresh process and after the others."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

MAX = 32 << 20


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2010_03090_gb300 as u
    return u.lib()


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
    return bufs


def test_noalloc_matches_host_entry_point(lib):
    for _ in range(2):  # two calls in a row on the same inputs
        for b in _inputs():
            p = b.ctypes.data_as(ctypes.c_void_p)
            want = lib.utf8_validate_host(p, b.size, None)
            assert lib.utf8_last_error() == 0
            got = lib.utf8_validate_host_noalloc(p, b.size, None)
            assert lib.utf8_last_error() == 0
            assert got == want, b.size


def test_noalloc_rejects_oversize(lib):
    b = np.zeros(MAX + 1, dtype=np.uint8)
    assert lib.utf8_validate_host_noalloc(b.ctypes.data_as(ctypes.c_void_p), b.size, None) is False
    assert lib.utf8_last_error() == 4  # UTF8_ERR_BUDGET
    assert lib.utf8_validate_host_noalloc(None, 0, None) is True
