"""Parity of the host-CPU `lookup` baseline (cpu_lookup/, 16-byte vectors)
with the oracle: exhaustive short strings, every class string of up to three
bytes placed across the 16- and 64-byte block edges (the ASCII early-out and
the previous-vector carry), injected errors at block edges, batches."""
import itertools

import numpy as np

import cpu_lookup
import oracle
import synth

REPS = [0x41, 0x85, 0x95, 0xA5, 0xC0, 0xC5, 0xE0, 0xE5, 0xED, 0xEE, 0xF0, 0xF2, 0xF4, 0xF8]


def test_every_short_string():
    for length in range(3):
        for t in itertools.product(range(256), repeat=length):
            b = bytes(t)
            assert cpu_lookup.valid(b) == oracle.valid(b), b.hex()
    for length in range(1, 5):
        for t in itertools.product(REPS, repeat=length):
            b = bytes(t)
            assert cpu_lookup.valid(b) == oracle.valid(b), b.hex()


def test_class_strings_across_block_edges():
    """ASCII before (so that 64-byte blocks are all ASCII) and after each
    class string, with the string straddling every position of a 64-byte
    block and of the last partial vector."""
    for pad in list(range(0, 20)) + list(range(44, 84)) + [125, 126, 127, 128, 129]:
        head = b"A" * pad
        for length in range(1, 4):
            for t in itertools.product(REPS, repeat=length):
                for tail in (b"", b"B" * (70 - pad % 64)):
                    b = head + bytes(t) + tail
                    assert cpu_lookup.valid(b) == oracle.valid(b), (pad, bytes(t).hex(), len(tail))


def test_injected_errors_at_block_edges():
    rng = np.random.default_rng(17)
    for model in (synth.UNIFORM, synth.CJK, synth.LATIN, synth.EMOJI):
        base = synth.fill(1 << 16, model, seed=model + 3)
        assert cpu_lookup.valid(base) and oracle.valid(base)
        for period in (16, 64, 4096):
            for k in (1, 5):
                for d in range(5):
                    buf = base.copy()
                    kind = synth.ERROR_CLASSES[int(rng.integers(0, 7))]
                    synth.inject_any(buf, kind, rng, at=k * period - d)
                    assert cpu_lookup.valid(buf) == oracle.valid(buf), (model, period, k, d, kind)


def test_workload_1mib():
    bufs, labels = synth.workload_1mib()
    assert [cpu_lookup.valid(b) for b in bufs] == [oracle.valid(b) for b in bufs], labels


def test_batch_matches_oracle():
    data, offsets, _ = synth.workload_batch_1m(count=20000, total=20000 * 537)
    want = oracle.valid_batch(data, offsets, threads=4)
    for threads in (1, 4):
        assert np.array_equal(cpu_lookup.valid_batch(data, offsets, threads=threads), want)
