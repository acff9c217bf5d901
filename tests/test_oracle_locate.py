"""Pins of the oracle's error location (oracle.locate / locate_batch).

The position is the length of the longest valid prefix; it is pinned by
Python's strict UTF-8 codec (UnicodeDecodeError.start is where the first
ill-formed sequence starts) and by brute force over prefixes with the
validity oracle.  The rule (Section 3, a-f numbered 1-6) is pinned by
construction: each class of bad character is built from its definition
(Table 1's bit layout, Python's surrogatepass encoder) after a valid prefix.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth

REPS = [0x41, 0x85, 0x95, 0xA5, 0xC0, 0xC5, 0xE0, 0xE5, 0xED, 0xEE, 0xF0, 0xF2, 0xF4, 0xF8]


def codec_position(b: bytes) -> int:
    try:
        b.decode("utf-8")
        return len(b)
    except UnicodeDecodeError as e:
        return e.start


def prefix_position(b: bytes) -> int:
    """Brute force: the largest m with b[:m] valid (validity oracle)."""
    return max(m for m in range(len(b) + 1) if oracle.valid(b[:m]))


def encode_form(cp: int, k: int) -> bytes:
    """Table 1's k-byte bit layout of cp, whether or not cp is allowed there."""
    if k == 2:
        return bytes([0xC0 | (cp >> 6), 0x80 | (cp & 0x3F)])
    if k == 3:
        return bytes([0xE0 | (cp >> 12), 0x80 | ((cp >> 6) & 0x3F), 0x80 | (cp & 0x3F)])
    return bytes([0xF0 | (cp >> 18), 0x80 | ((cp >> 12) & 0x3F), 0x80 | ((cp >> 6) & 0x3F),
                  0x80 | (cp & 0x3F)])


def random_text(rng, chars: int) -> bytes:
    out = []
    for _ in range(chars):
        k = int(rng.integers(1, 5))
        lo, hi = [(0, 0x7F), (0x80, 0x7FF), (0x800, 0xFFFF), (0x10000, 0x10FFFF)][k - 1]
        cp = int(rng.integers(lo, hi + 1))
        if 0xD800 <= cp <= 0xDFFF:
            cp = 0x41
        out.append(chr(cp).encode("utf-8"))
    return b"".join(out)


def bad_character(rule: int, rng) -> bytes:
    """A character that breaks exactly `rule` (1-6), as its definition says."""
    if rule == 1:    # a: five or more header bits
        return bytes([int(rng.integers(0xF8, 0x100))])
    if rule == 2:    # b: a valid character cut short
        full = chr(int(rng.integers(0x80, 0x110000)) if rng.random() < 0.9 else 0x20AC)
        try:
            enc = full.encode("utf-8")
        except UnicodeEncodeError:  # a surrogate was drawn
            enc = "€".encode("utf-8")
        return enc[:int(rng.integers(1, len(enc)))] if len(enc) > 1 else b"\xc3"
    if rule == 3:    # c: a continuation byte where a character starts
        return bytes([int(rng.integers(0x80, 0xC0))])
    if rule == 4:    # d: overlong forms
        k = int(rng.integers(2, 5))
        limit = {2: 0x80, 3: 0x800, 4: 0x10000}[k]
        return encode_form(int(rng.integers(0, limit)), k)
    if rule == 5:    # e: above U+10FFFF in the 4-byte layout
        return encode_form(int(rng.integers(0x110000, 0x200000)), 4)
    return chr(int(rng.integers(0xD800, 0xE000))).encode("utf-8", "surrogatepass")  # f


def test_encode_form_matches_python_on_valid_code_points():
    for cp in (0x80, 0x7FF, 0x800, 0xFFFF, 0x10000, 0x10FFFF, 0x20AC, 0x1F600):
        k = len(chr(cp).encode("utf-8"))
        assert encode_form(cp, k) == chr(cp).encode("utf-8")


def test_position_matches_codec_on_all_short_byte_strings():
    for length in range(3):
        for t in itertools.product(range(256), repeat=length):
            b = bytes(t)
            pos, rule = oracle.locate(b)
            assert pos == codec_position(b), b.hex()
            assert (rule == 0) == (pos == len(b)) == oracle.valid(b)


def test_position_matches_codec_and_brute_force_on_class_strings():
    for length in range(1, 5):
        for t in itertools.product(REPS, repeat=length):
            b = bytes(t)
            pos, _ = oracle.locate(b)
            assert pos == codec_position(b) == prefix_position(b), b.hex()


@pytest.mark.parametrize("rule", range(1, 7))
def test_rule_by_construction(rule):
    rng = np.random.default_rng(100 + rule)
    for _ in range(400):
        head = random_text(rng, int(rng.integers(0, 12)))
        bad = bad_character(rule, rng)
        if rule == 2:   # what follows a cut character must not continue it
            tail = random_text(rng, int(rng.integers(0, 6))) if rng.random() < 0.8 else b""
        else:
            tail = bytes(rng.integers(0, 256, int(rng.integers(0, 8)), dtype=np.uint8))
        b = head + bad + tail
        assert oracle.locate(b) == (len(head), rule), (head.hex(), bad.hex(), tail.hex())
        assert codec_position(b) == len(head)


def test_injected_errors_in_large_buffers():
    """The synthetic corruptions (one per class, mid-buffer): the codec and
    the oracle agree on where the first error starts."""
    rng = np.random.default_rng(5)
    base = synth.fill(1 << 16, synth.UNIFORM, seed=21)
    assert oracle.locate(base) == (base.size, 0)
    for kind in synth.ERROR_CLASSES:
        b = base.copy()
        synth.inject_any(b, kind, rng)
        pos, rule = oracle.locate(b)
        assert 1 <= rule <= 6
        assert pos == codec_position(b.tobytes())


def test_batch_matches_single():
    rng = np.random.default_rng(9)
    strings = []
    for k in range(3000):
        s = random_text(rng, int(rng.integers(0, 20)))
        if k % 3 == 0 and s:
            s = s + bad_character(int(rng.integers(1, 7)), rng) + random_text(rng, 2)
        strings.append(s)
    offsets = np.cumsum([0] + [len(s) for s in strings]).astype(np.int64)
    data = np.frombuffer(b"".join(strings) or b"\0", np.uint8)
    for threads in (1, 4):
        pos, rule = oracle.locate_batch(data, offsets, threads=threads)
        for k, s in enumerate(strings):
            assert (pos[k], rule[k]) == oracle.locate(s)
